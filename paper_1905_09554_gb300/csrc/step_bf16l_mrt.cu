// Step kernels for CodecBF16Local storage with the COLL_MRT collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(bf16l_mrt, CodecBF16Local, COLL_MRT, false)
