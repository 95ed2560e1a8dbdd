// Step kernels for CodecBF16Local storage with the COLL_SRT collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(bf16l_srt, CodecBF16Local, COLL_SRT, false)
