// Step kernels for CodecF32 storage with the COLL_SRT collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f32_srt, CodecF32, COLL_SRT, true)
