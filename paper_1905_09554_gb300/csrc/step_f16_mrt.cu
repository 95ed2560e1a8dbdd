// Step kernels for CodecF16Dev storage with the COLL_MRT collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f16_mrt, CodecF16Dev, COLL_MRT, false)
