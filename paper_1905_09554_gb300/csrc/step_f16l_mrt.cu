// Step kernels for CodecF16Local storage with the COLL_MRT collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f16l_mrt, CodecF16Local, COLL_MRT, false)
