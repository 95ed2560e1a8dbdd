// Step kernels for CodecBF16Dev storage with the COLL_MRT collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(bf16_mrt, CodecBF16Dev, COLL_MRT, false)
