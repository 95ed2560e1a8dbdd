// Step kernels for CodecF64 storage with the COLL_MRT_UNIT collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f64_mrtu, CodecF64, COLL_MRT_UNIT, true)
