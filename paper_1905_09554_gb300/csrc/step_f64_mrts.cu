// Step kernels for CodecF64 storage with the COLL_MRT_SPARSE collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f64_mrts, CodecF64, COLL_MRT_SPARSE, true)
