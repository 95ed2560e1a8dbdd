// Step kernels for CodecBF16Dev storage with the COLL_MRT_UNIT collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(bf16_mrtu, CodecBF16Dev, COLL_MRT_UNIT, false)
