// Step kernels for CodecBF16Dev storage with the COLL_SRT collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(bf16_srt, CodecBF16Dev, COLL_SRT, false)
