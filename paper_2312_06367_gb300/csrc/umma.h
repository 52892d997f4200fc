// BF16x3 split-precision tensor-core (tcgen05 / TMEM / TMA) path of the history sum.
#pragma once
#include "internal.h"

namespace tdc {
struct StepPlan;
struct Bf16x3Gemm;
tdcfie_status build_bf16x3(tdcfie_t h, StepPlan* p);
void launch_step_bf16x3(tdcfie_t h, StepPlan* p, cudaStream_t s);
void destroy_bf16x3(Bf16x3Gemm* g);
cudaError_t reset_bf16x3(Bf16x3Gemm* g, int ring, cudaStream_t s);
}  // namespace tdc
