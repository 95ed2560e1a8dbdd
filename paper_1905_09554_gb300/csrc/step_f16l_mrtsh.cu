// Step kernels for CodecF16Local storage with the COLL_MRT_SHEAR collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(f16l_mrtsh, CodecF16Local, COLL_MRT_SHEAR, false)
