// Restarted mixed-precision GMRES on T_0 (per-step solve of the MOT recurrence).
#pragma once
#include "internal.h"

namespace tdc {
struct StepPlan;
struct GmresPlan;
cudaError_t build_gmres(tdcfie_t h, StepPlan* p);
void destroy_gmres(GmresPlan* g);
cudaError_t reset_gmres_stats(GmresPlan* g);
void gmres_set_tol(GmresPlan* g, double tol);
// out6: Arnoldi iterations, steps, max per step, this step, solves not converged, loop passes
cudaError_t gmres_stats(GmresPlan* g, long long* out6);
int gmres_body_launches();
// b: right-hand side (path type, R x ne); learned: learned guess buffer (or nullptr); T0p: T_0 in the
// path precision; the solution goes to ring slot n % ring.  s must be capturing a graph.
template <typename T>
cudaError_t launch_gmres(tdcfie_t h, StepPlan* p, const T* b, const T* learned, const T* T0p, T* ringbuf, cudaStream_t s);

// Learned initial guess (mlp.cu): FP16 weights on the device, filled into p->guessbuf each step.
struct MlpState;
cudaError_t build_mlp(StepPlan* p);
void destroy_mlp(MlpState* m);
cudaError_t mlp_load(StepPlan* p, const float* host_params, cudaStream_t s);
template <typename T>
void launch_mlp_guess(StepPlan* p, cudaStream_t s);
}  // namespace tdc
