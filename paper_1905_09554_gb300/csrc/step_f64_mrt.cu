// Step kernels for CodecF64 storage with the COLL_MRT collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f64_mrt, CodecF64, COLL_MRT, true)
