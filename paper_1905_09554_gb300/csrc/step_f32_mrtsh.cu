// Step kernels for CodecF32 storage with the COLL_MRT_SHEAR collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f32_mrtsh, CodecF32, COLL_MRT_SHEAR, true)
