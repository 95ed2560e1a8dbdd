// Step kernels for CodecBF16Local storage with the COLL_MRT_SHEAR collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(bf16l_mrtsh, CodecBF16Local, COLL_MRT_SHEAR, false)
