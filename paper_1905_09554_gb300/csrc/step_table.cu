// Table of the step kernels by (storage, collision).
#include "step_args.h"

namespace lbm {

extern const StepKernels kStep_f64_srt;
extern const StepKernels kStep_f64_mrt;
extern const StepKernels kStep_f64_mrts;
extern const StepKernels kStep_f64_mrtu;
extern const StepKernels kStep_f64_mrtsh;
extern const StepKernels kStep_f32_srt;
extern const StepKernels kStep_f32_mrt;
extern const StepKernels kStep_f32_mrts;
extern const StepKernels kStep_f32_mrtu;
extern const StepKernels kStep_f32_mrtsh;
extern const StepKernels kStep_f16_srt;
extern const StepKernels kStep_f16_mrt;
extern const StepKernels kStep_f16_mrts;
extern const StepKernels kStep_f16_mrtu;
extern const StepKernels kStep_f16_mrtsh;
extern const StepKernels kStep_bf16_srt;
extern const StepKernels kStep_bf16_mrt;
extern const StepKernels kStep_bf16_mrts;
extern const StepKernels kStep_bf16_mrtu;
extern const StepKernels kStep_bf16_mrtsh;
extern const StepKernels kStep_f16l_srt;
extern const StepKernels kStep_f16l_mrt;
extern const StepKernels kStep_f16l_mrts;
extern const StepKernels kStep_f16l_mrtu;
extern const StepKernels kStep_f16l_mrtsh;
extern const StepKernels kStep_bf16l_srt;
extern const StepKernels kStep_bf16l_mrt;
extern const StepKernels kStep_bf16l_mrts;
extern const StepKernels kStep_bf16l_mrtu;
extern const StepKernels kStep_bf16l_mrtsh;

const StepKernels& step_kernels(int storage, int coll) {
    static const StepKernels* table[6][COLL_COUNT] = {
        {&kStep_f64_srt, &kStep_f64_mrt, &kStep_f64_mrts, &kStep_f64_mrtu, &kStep_f64_mrtsh},
        {&kStep_f32_srt, &kStep_f32_mrt, &kStep_f32_mrts, &kStep_f32_mrtu, &kStep_f32_mrtsh},
        {&kStep_f16_srt, &kStep_f16_mrt, &kStep_f16_mrts, &kStep_f16_mrtu, &kStep_f16_mrtsh},
        {&kStep_bf16_srt, &kStep_bf16_mrt, &kStep_bf16_mrts, &kStep_bf16_mrtu, &kStep_bf16_mrtsh},
        {&kStep_f16l_srt, &kStep_f16l_mrt, &kStep_f16l_mrts, &kStep_f16l_mrtu, &kStep_f16l_mrtsh},
        {&kStep_bf16l_srt, &kStep_bf16l_mrt, &kStep_bf16l_mrts, &kStep_bf16l_mrtu, &kStep_bf16l_mrtsh},
    };
    return *table[storage][coll];
}

}  // namespace lbm
