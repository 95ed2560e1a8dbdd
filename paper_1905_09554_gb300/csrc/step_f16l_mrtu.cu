// Step kernels for CodecF16Local storage with the COLL_MRT_UNIT collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f16l_mrtu, CodecF16Local, COLL_MRT_UNIT, false)
