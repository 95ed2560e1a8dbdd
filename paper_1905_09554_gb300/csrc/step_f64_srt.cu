// Step kernels for CodecF64 storage with the COLL_SRT collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f64_srt, CodecF64, COLL_SRT, true)
