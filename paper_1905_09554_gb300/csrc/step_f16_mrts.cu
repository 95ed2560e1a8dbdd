// Step kernels for CodecF16Dev storage with the COLL_MRT_SPARSE collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f16_mrts, CodecF16Dev, COLL_MRT_SPARSE, false)
