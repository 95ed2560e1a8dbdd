// Step kernels for CodecF32 storage with the COLL_MRT_UNIT collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f32_mrtu, CodecF32, COLL_MRT_UNIT, true)
