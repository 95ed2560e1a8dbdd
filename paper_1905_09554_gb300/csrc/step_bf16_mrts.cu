// Step kernels for CodecBF16Dev storage with the COLL_MRT_SPARSE collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(bf16_mrts, CodecBF16Dev, COLL_MRT_SPARSE, false)
