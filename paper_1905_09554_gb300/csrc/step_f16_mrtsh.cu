// Step kernels for CodecF16Dev storage with the COLL_MRT_SHEAR collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f16_mrtsh, CodecF16Dev, COLL_MRT_SHEAR, false)
