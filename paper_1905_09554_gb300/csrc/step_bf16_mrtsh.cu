// Step kernels for CodecBF16Dev storage with the COLL_MRT_SHEAR collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(bf16_mrtsh, CodecBF16Dev, COLL_MRT_SHEAR, false)
