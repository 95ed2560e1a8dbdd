// Step kernel instantiations for CodecBF16Dev storage.
#include "step_dispatch.cuh"

namespace lbm {

cudaError_t launch_step_bf16(const StepLaunch& l, const void* src, void* dst) {
    return launch_step_s<CodecBF16Dev>(l, src, dst);
}

int prepare_step_bf16(const StepLaunch& l) { return prepare_async_s<CodecBF16Dev>(l); }

}  // namespace lbm
