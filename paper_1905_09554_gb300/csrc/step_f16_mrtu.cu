// Step kernels for CodecF16Dev storage with the COLL_MRT_UNIT collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f16_mrtu, CodecF16Dev, COLL_MRT_UNIT, false)
