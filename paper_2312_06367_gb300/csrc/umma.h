// Split-precision tensor-core (tcgen05 / TMEM / TMA) step of the MOT recurrence (FP16X3, BF16X3) and
// the stand-alone split-precision product behind tdcfie_tc_gemm.
#pragma once
#include "internal.h"

namespace tdc {
struct StepPlan;
struct TcStep;
tdcfie_status build_tc(tdcfie_t h, StepPlan* p);
void launch_step_tc(tdcfie_t h, StepPlan* p, cudaStream_t s);
void destroy_tc(TcStep* g);
cudaError_t reset_tc(TcStep* g, int ring, int ne, cudaStream_t s);
tdcfie_status tc_gemm(int precision, const double* blocks, int64_t nblk, int64_t rows, int64_t cols, const double* x,
                      int64_t R, double* out, cudaStream_t s);
}  // namespace tdc
