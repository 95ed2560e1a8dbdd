// Step kernels for CodecF32 storage with the COLL_MRT collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f32_mrt, CodecF32, COLL_MRT, true)
