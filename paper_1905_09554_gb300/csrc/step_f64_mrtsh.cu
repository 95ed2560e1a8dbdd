// Step kernels for CodecF64 storage with the COLL_MRT_SHEAR collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f64_mrtsh, CodecF64, COLL_MRT_SHEAR, true)
