// Step kernels for CodecF16Dev storage with the COLL_SRT collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f16_srt, CodecF16Dev, COLL_SRT, false)
