// Step kernels for CodecBF16Local storage with the COLL_MRT_SPARSE collision.
#include "step_dispatch.cuh"

LBM_STEP_INSTANCE(bf16l_mrts, CodecBF16Local, COLL_MRT_SPARSE, false)
