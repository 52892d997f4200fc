// Several scatterers marched together: one CUDA graph holds one step of every handle, each on its
// own forked stream, so a single graph launch advances all of them and their kernels run
// concurrently (uneven sizes fill the GPU together instead of one after another).  The handles keep
// their own blocks, rings and step counters; the arithmetic per handle is exactly that of
// tdcfie_step.
#include <string>
#include <vector>

#include "internal.h"
#include "plan.h"

using namespace tdc;

struct tdcfie_batch_s {
    std::vector<tdcfie_t> hs;
    cudaStream_t main = nullptr;
    std::vector<cudaStream_t> branch;
    std::vector<cudaEvent_t> joined;
    cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double last_step_ms = 0.0;
    int64_t launches_per_step = 0;
};

static void destroy_batch(tdcfie_batch_t b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto s : b->branch) cudaStreamDestroy(s);
    for (auto e : b->joined) cudaEventDestroy(e);
    for (cudaEvent_t e : {b->fork, b->t0, b->t1})
        if (e) cudaEventDestroy(e);
    if (b->main) cudaStreamDestroy(b->main);
    delete b;
}

#define BK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { destroy_batch(b); return cuda_fail(nullptr, e_, #x); } } while (0)

extern "C" tdcfie_status tdcfie_batch_create(const tdcfie_t* handles, int64_t n, tdcfie_batch_t* out) {
    if (!handles || !out || n < 1) return fail(nullptr, TDCFIE_E_ARG, "need n >= 1 handles and an output pointer");
    if (n > 4096) return fail(nullptr, TDCFIE_E_ARG, "at most 4096 handles in a batch");
    for (int64_t i = 0; i < n; ++i) {
        if (!handles[i]) return fail(nullptr, TDCFIE_E_ARG, "NULL handle in the batch");
        if (!handles[i]->assembled || !handles[i]->plan)
            return fail(nullptr, TDCFIE_E_STATE, "every handle must be assembled before tdcfie_batch_create");
        if (handles[i]->opts.device != handles[0]->opts.device)
            return fail(nullptr, TDCFIE_E_ARG, "all handles of a batch must use the same device");
        for (int64_t j = 0; j < i; ++j)
            if (handles[j] == handles[i]) return fail(nullptr, TDCFIE_E_ARG, "a handle appears twice in the batch");
    }
    auto* b = new tdcfie_batch_s();
    b->hs.assign(handles, handles + n);
    BK(cudaSetDevice(handles[0]->opts.device));
    BK(cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking));
    BK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    BK(cudaEventCreate(&b->t0));
    BK(cudaEventCreate(&b->t1));
    for (int64_t i = 0; i < n; ++i) {
        cudaStream_t s;
        cudaEvent_t e;
        BK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        b->branch.push_back(s);
        BK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->joined.push_back(e);
    }
    *out = b;
    return TDCFIE_OK;
}

extern "C" tdcfie_status tdcfie_batch_step(tdcfie_batch_t b, int64_t nsteps, void* const* currents_out) {
    if (!b) return fail(nullptr, TDCFIE_E_ARG, "batch is NULL");
    if (nsteps < 0) return fail(nullptr, TDCFIE_E_ARG, "nsteps < 0");
    const int64_t n = (int64_t)b->hs.size();
    for (tdcfie_t h : b->hs)
        if (!h->excited || !h->plan)
            return fail(nullptr, TDCFIE_E_STATE, "set the excitation of every handle of the batch first");
    if (nsteps == 0) return TDCFIE_OK;
    cudaError_t e = cudaSetDevice(b->hs[0]->opts.device);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
    for (int64_t i = 0; i < n; ++i) {
        const tdcfie_status st = plan_set_outputs(b->hs[i], currents_out ? currents_out[i] : nullptr, nullptr);
        if (st != TDCFIE_OK) return fail(nullptr, st, "batch handle " + std::to_string(i) + ": " + b->hs[i]->err);
    }
    if (!b->exec) {
        // one step of every handle, each on its own branch of the graph
        e = cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaStreamBeginCapture");
        cudaError_t ce = cudaEventRecord(b->fork, b->main);
        b->launches_per_step = 0;
        for (int64_t i = 0; i < n && ce == cudaSuccess; ++i) {
            ce = cudaStreamWaitEvent(b->branch[i], b->fork, 0);
            if (ce == cudaSuccess) ce = capture_step(b->hs[i], b->branch[i]);
            if (ce == cudaSuccess) ce = cudaEventRecord(b->joined[i], b->branch[i]);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->main, b->joined[i], 0);
            b->launches_per_step += plan_launches_per_step(b->hs[i]);
        }
        const cudaError_t ee = cudaStreamEndCapture(b->main, &b->graph);
        if (ce != cudaSuccess || ee != cudaSuccess) {
            if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
            return cuda_fail(nullptr, ce != cudaSuccess ? ce : ee, "capturing the batch step graph");
        }
        e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGraphInstantiate (batch)");
    }
    e = cudaEventRecord(b->t0, b->main);
    for (int64_t i = 0; i < nsteps && e == cudaSuccess; ++i) e = cudaGraphLaunch(b->exec, b->main);
    if (e == cudaSuccess) e = cudaEventRecord(b->t1, b->main);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->main);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch step");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->t0, b->t1);
    b->last_step_ms = ms / (double)nsteps;
    for (int64_t i = 0; i < n; ++i) {
        const tdcfie_status st = plan_check(b->hs[i]);
        if (st != TDCFIE_OK) return fail(nullptr, st, "batch handle " + std::to_string(i) + ": " + b->hs[i]->err);
    }
    return TDCFIE_OK;
}

extern "C" tdcfie_status tdcfie_batch_timing(tdcfie_batch_t b, double* step_ms, int64_t* launches_per_step) {
    if (!b) return fail(nullptr, TDCFIE_E_ARG, "batch is NULL");
    if (step_ms) *step_ms = b->last_step_ms;
    if (launches_per_step) *launches_per_step = b->launches_per_step;
    return TDCFIE_OK;
}

extern "C" tdcfie_status tdcfie_batch_destroy(tdcfie_batch_t b) {
    destroy_batch(b);
    return TDCFIE_OK;
}
