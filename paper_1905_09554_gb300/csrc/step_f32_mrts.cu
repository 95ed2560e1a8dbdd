// Step kernels for CodecF32 storage with the COLL_MRT_SPARSE collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f32_mrts, CodecF32, COLL_MRT_SPARSE, true)
