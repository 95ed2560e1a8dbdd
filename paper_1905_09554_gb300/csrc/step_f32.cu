// Step kernel instantiations for CodecF32 storage.
#include "step_dispatch.cuh"

namespace lbm {

cudaError_t launch_step_f32(const StepLaunch& l, const void* src, void* dst) {
    return launch_step_s<CodecF32>(l, src, dst);
}

int prepare_step_f32(const StepLaunch& l) { return prepare_async_s<CodecF32>(l); }

cudaError_t launch_batch_step_f32(const StepLaunch& l, const BatchArgs& b, const void* src, void* dst) {
    return launch_batch_s<CodecF32>(l, b, src, dst);
}

int prepare_batch_step_f32(const StepLaunch& l) { return prepare_batch_s<CodecF32>(l); }

}  // namespace lbm
