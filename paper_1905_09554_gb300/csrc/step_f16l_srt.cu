// Step kernels for CodecF16Local storage with the COLL_SRT collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f16l_srt, CodecF16Local, COLL_SRT, false)
