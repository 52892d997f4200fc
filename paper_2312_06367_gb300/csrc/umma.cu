// BF16x3 tensor-core history sum (placeholder until the tcgen05 kernel lands).
#include "umma.h"

namespace tdc {
struct Bf16x3Gemm {};
tdcfie_status build_bf16x3(tdcfie_t h, StepPlan*) {
    return fail(h, TDCFIE_E_UNSUPPORTED, "BF16X3 path not built yet");
}
void launch_step_bf16x3(tdcfie_t, StepPlan*, cudaStream_t) {}
void destroy_bf16x3(Bf16x3Gemm* g) { delete g; }
}  // namespace tdc
