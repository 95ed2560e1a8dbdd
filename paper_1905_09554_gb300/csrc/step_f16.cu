// Step kernel instantiations for CodecF16Dev storage.
#include "step_dispatch.cuh"

namespace lbm {

cudaError_t launch_step_f16(const StepLaunch& l, const void* src, void* dst) {
    return launch_step_s<CodecF16Dev>(l, src, dst);
}

int prepare_step_f16(const StepLaunch& l) { return prepare_async_s<CodecF16Dev>(l); }

}  // namespace lbm
