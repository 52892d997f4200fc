// Per-handle step plan shared by the SIMT (march.cu) and tensor-core (umma.cu) paths.
#pragma once
#include <vector>

#include "internal.h"

namespace tdc {
struct TcStep;
struct GmresPlan;
struct MlpState;
struct FactPlan;

struct StepPlan {
    int prec = TDCFIE_FP64;
    int R = 1, ne = 0, nc = 0, K = 0, nblk = 0, ring = 0;
    size_t esz = 8;
    void* blocks = nullptr;      // nblk x ne x ne (path precision): -A, alpha L2, -T_1 .. -T_{K-1}
    void* t0inv = nullptr;       // ne x ne
    void* t0mat = nullptr;       // ne x ne, T_0 itself (GMRES matvec)
    void* guessbuf = nullptr;    // R x ne learned initial guess
    GmresPlan* gm = nullptr;
    MlpState* mlp = nullptr;     // learned-guess network (GMRES with TDCFIE_GUESS_MLP)
    bool gmres_on = false;       // per-step solve by GMRES (else the explicit T_0^-1)
    bool mlp_on = false;         // learned guess evaluated each step
    bool guess_extrap = false;   // learned guess on top of the cubic extrapolation (else y_{n-1})
    void* pinv = nullptr;        // nc x nc
    void* E = nullptr;           // R x ne  (e_n)
    void* Hv = nullptr;          // R x ne  (h_n)
    void* ringbuf = nullptr;     // ring x R x ne
    void* b = nullptr;           // R x ne
    void* partial = nullptr;     // nblk x R x ne
    void* w = nullptr;           // R x ne
    void* z = nullptr;           // R x nc
    void* u = nullptr;           // R x nc
    const void** xptr = nullptr; // device array (unused for SIMT: computed in kernel)
    Ctl* ctl = nullptr;
    // rhs tables: per edge, quadrature points (x) and weighted basis vectors (c), e-points first
    int* pptr = nullptr; int* pnE = nullptr; void* px = nullptr; void* pc = nullptr;
    // factored history form (factored.cu); blocks and t0inv are then unused
    FactPlan* fact = nullptr;
    // tensor-core path
    TcStep* gemm = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
    cudaEvent_t evA = nullptr, evB = nullptr;            // captured around the history sum
    cudaGraphNode_t nodeA = nullptr, nodeB = nullptr;    // their record nodes in the step graph
    std::vector<cudaEvent_t> hA, hB;                     // per-step events of a tdcfie_step call
    int launches_per_step = 0;
};

// plane-wave tests e_n, h_n of one step into p.E, p.Hv (march.cu)
template <typename T>
void launch_rhs(tdcfie_t h, StepPlan& p, cudaStream_t s);
// factored history form (factored.cu)
tdcfie_status build_fact(tdcfie_t h, StepPlan* p);
tdcfie_status reset_fact(tdcfie_t h, StepPlan* p);
void destroy_fact(FactPlan* f);
double fact_step_bytes(const StepPlan* p);
int64_t fact_nnz(const StepPlan* p, bool stored);
template <typename T>
cudaError_t launch_step_fact(tdcfie_t h, StepPlan& p, cudaStream_t s);

}  // namespace tdc
