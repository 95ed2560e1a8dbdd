// Step kernel instantiations for CodecF32 storage.
#include "step_dispatch.cuh"

namespace lbm {

cudaError_t launch_step_f32(const StepLaunch& l, const void* src, void* dst) {
    return launch_step_s<CodecF32>(l, src, dst);
}

int prepare_step_f32(const StepLaunch& l) { return prepare_async_s<CodecF32>(l); }

}  // namespace lbm
