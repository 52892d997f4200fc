// Several scatterers marched together (the uneven batch).  Two forms, chosen at creation:
//
//  * Persistent (every member FP32, one incident wave, direct solve: the uneven-batch workload):
//    ONE cooperative kernel per step walks a work list of all members' items -- plane-wave tests
//    (32 edges), history partial sums (BCH rows of BQ blocks, into the member's per-block partial
//    buffer), their reduction over the blocks in block order (32 edges), T_0^-1 rows, projector
//    gathers (32 triangles), pseudo-inverse rows, post-processing (32 edges) -- with grid-wide
//    barriers between the seven phases.  Warps take items from a per-phase counter; the items are listed
//    longest first, so big scatterers start early and small ones fill the tail.  The row dot
//    products use the same arithmetic as the per-handle step (simt.h), so every member's
//    currents equal those of tdcfie_step bit for bit.  Rows per warp, warps per block and blocks
//    per SM come from a measuring autotuner (tdcfie_batch_tune).
//  * Graph branches (any other mix of precisions, waves or solvers): one CUDA graph holds one step
//    of every handle, each on its own forked stream.
// Either way a single graph launch advances all members; the handles keep their own blocks,
// rings and step counters.  Every grid-wide wait is bounded (%globaltimer, 2 s) and reports
// TDCFIE_E_TIMEOUT.
#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"
#include "plan.h"
#include "simt.h"

using namespace tdc;

namespace tdc {

struct BMember {            // device view of one member handle (FP32, one wave)
    int ne, nc, nblk, ring;
    const float* blocks;    // nblk x ne x ne: -A, alpha L2, -T_1 .. -T_{K-1}
    const float* t0inv;     // ne x ne
    const float* pinv;      // nc x nc
    float *E, *H, *ringbuf, *b, *z, *u;
    double* partial;        // nblk x ne per-block history sums
    const int* pptr;
    const int* pnE;
    const float* px;
    const float* pc;
    const double* exc;
    DevMesh m;
    double dt, dtt;
    Ctl* ctl;
};

struct BItem {
    int member, first, count, block;   // block: first block of a history item (else 0)
};

enum { PH_RHS = 0, PH_HIST, PH_RED, PH_SOLVE, PH_PIN, PH_PINV, PH_POUT, NPH };
constexpr int BCH = 8;                 // rows per work item of the row phases
constexpr int BQ = 4;                  // blocks per history work item
constexpr uint64_t BWAIT_NS = 2000000000ull;

struct BArgs {
    const BMember* mem;
    int nmem;
    const BItem* items[NPH];
    int nitems[NPH];
    unsigned* sync;     // [NPH] take counters, arrival count, generation, timeout flag
};

__device__ __forceinline__ uint64_t bclock() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// grid-wide barrier of the co-resident blocks (cooperative launch); bounded spin
__device__ __forceinline__ void grid_barrier(unsigned* sync) {
    unsigned* count = sync + NPH;
    volatile unsigned* gen = sync + NPH + 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(count, 1u) == gridDim.x - 1) {
            *count = 0;
            __threadfence();
            atomicAdd(sync + NPH + 1, 1u);
        } else {
            const uint64_t t0 = bclock();
            while (*gen == g) {
                if (bclock() - t0 > BWAIT_NS) {
                    atomicExch(sync + NPH + 2, 1u);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// acc[i] = B_i . x for the nrows (<= ROWS) rows B_i = B0 + i ld of one warp, R = 1; the per-row
// arithmetic is that of RowDot<float, 1> (four compensated lanes accumulators, FP64 combination),
// but each float4 of x is loaded once for all rows
template <int ROWS>
__device__ __forceinline__ void rows_dot(const float* __restrict__ B0, int64_t ld, int nrows, int ncols,
                                         const float* __restrict__ x, double* acc) {
    const bool vec = ((ncols | (int)ld) & 3) == 0 &&
                     ((reinterpret_cast<uintptr_t>(B0) | reinterpret_cast<uintptr_t>(x)) & 15) == 0;
    if (!vec) {
        for (int i = 0; i < nrows; ++i) RowDot<float, 1>::run(B0 + i * ld, ncols, x, 1, ncols, acc + i);
        return;
    }
    const int lane = threadIdx.x & 31;
    float hi[ROWS][4], lo[ROWS][4];
#pragma unroll
    for (int i = 0; i < ROWS; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) hi[i][c] = lo[i][c] = 0.f;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    for (int j = lane; j < (ncols >> 2); j += 32) {
        const float4 v = x4[j];
#pragma unroll
        for (int i = 0; i < ROWS; ++i)
            if (i < nrows) {
                const float4 a = reinterpret_cast<const float4*>(B0 + i * ld)[j];
                ff_add(hi[i][0], lo[i][0], a.x, v.x);
                ff_add(hi[i][1], lo[i][1], a.y, v.y);
                ff_add(hi[i][2], lo[i][2], a.z, v.z);
                ff_add(hi[i][3], lo[i][3], a.w, v.w);
            }
    }
#pragma unroll
    for (int i = 0; i < ROWS; ++i) {
        double v = 0.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) v += (double)hi[i][c] + (double)lo[i][c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (i < nrows) acc[i] = v;
    }
}

template <int ROWS>
__device__ __forceinline__ void batch_item(int phase, const BMember& M, const BItem& it) {
    const int lane = threadIdx.x & 31;
    const int64_t n = M.ctl->n;
    const int ne = M.ne;
    float* yn = M.ringbuf + (n % M.ring) * (int64_t)ne;
    if (phase == PH_RHS) {
        const int e = it.first + lane;
        if (lane < it.count) {
            float ev, hv;
            rhs_edge<float>(M.exc, n, M.dt, e, M.pptr, M.px, M.pc, M.pnE, ev, hv);
            M.E[e] = ev;
            M.H[e] = hv;
        }
    } else if (phase == PH_HIST) {
        // per-block partial sums (the arithmetic of k_history_rows), reduced in block order by PH_RED
        const int q1 = min(M.nblk, it.block + BQ);
        for (int q = it.block; q < q1; ++q) {
            const float* x;
            if (q == 0) x = M.E;
            else if (q == 1) x = M.H;
            else {
                int64_t slot = (n - (q - 1)) % M.ring;
                if (slot < 0) slot += M.ring;
                x = M.ringbuf + slot * (int64_t)ne;
            }
            for (int r0 = it.first; r0 < it.first + it.count; r0 += ROWS) {
                const int nr = min(ROWS, it.first + it.count - r0);
                double acc[ROWS];
                rows_dot<ROWS>(M.blocks + ((int64_t)q * ne + r0) * ne, ne, nr, ne, x, acc);
                if (lane == 0)
                    for (int i = 0; i < nr; ++i) M.partial[(int64_t)q * ne + r0 + i] = acc[i];
            }
        }
    } else if (phase == PH_RED) {
        const int e = it.first + lane;
        if (lane < it.count) {
            double v = 0.0;
            for (int q = 0; q < M.nblk; ++q) v += M.partial[(int64_t)q * ne + e];
            M.b[e] = (float)v;
        }
    } else if (phase == PH_SOLVE || phase == PH_PINV) {
        const bool solve = phase == PH_SOLVE;
        const int cols = solve ? ne : M.nc;
        const float* Mx = solve ? M.t0inv : M.pinv;
        const float* x = solve ? M.b : M.z;
        float* dst = solve ? yn : M.u;
        for (int r0 = it.first; r0 < it.first + it.count; r0 += ROWS) {
            const int nr = min(ROWS, it.first + it.count - r0);
            double acc[ROWS];
            rows_dot<ROWS>(Mx + (int64_t)r0 * cols, cols, nr, cols, x, acc);
            if (lane == 0)
                for (int i = 0; i < nr; ++i) dst[r0 + i] = (float)acc[i];
        }
    } else if (phase == PH_PIN) {
        const int c = it.first + lane;
        if (lane < it.count) {
            const float* yp = M.ringbuf + ((n - 1) % M.ring) * (int64_t)ne;
            M.z[c] = (float)project_in_value<float>(M.m, c, yn, yp, n == 1, M.dtt);
        }
    } else {   // PH_POUT
        const int e = it.first + lane;
        if (lane < it.count) {
            const float val = yn[e] + M.u[M.m.cplus_[e]] - M.u[M.m.cminus_[e]];
            Ctl* ctl = M.ctl;
            if (!isfinite((double)val) && atomicCAS(&ctl->status, 0, (int)TDCFIE_E_NONFINITE) == 0) ctl->bad_step = n;
            if (ctl->out) reinterpret_cast<float*>(ctl->out)[(n - ctl->n0) * (int64_t)ne + e] = val;
            if (ctl->yout) reinterpret_cast<float*>(ctl->yout)[(n - ctl->n0) * (int64_t)ne + e] = yn[e];
        }
    }
}

// one MOT step of every member: seven phases over the work lists, grid barriers in between
template <int ROWS>
__global__ void k_batch_step(BArgs a) {
    const int lane = threadIdx.x & 31;
    for (int ph = 0; ph < NPH; ++ph) {
        const BItem* items = a.items[ph];
        const int nitems = a.nitems[ph];
        for (;;) {
            int i = 0;
            if (lane == 0) i = (int)atomicAdd(a.sync + ph, 1u);
            i = __shfl_sync(0xffffffffu, i, 0);
            if (i >= nitems) break;
            const BItem it = items[i];
            batch_item<ROWS>(ph, a.mem[it.member], it);
        }
        grid_barrier(a.sync);
    }
    // every block has passed the last barrier: advance the members and rearm the counters
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int s = 0; s < a.nmem; ++s) a.mem[s].ctl->n += 1;
        for (int ph = 0; ph < NPH; ++ph) a.sync[ph] = 0;
        __threadfence();
    }
}

}  // namespace tdc

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
    // persistent form
    bool persistent = false;
    BMember* dmem = nullptr;
    BItem* ditems = nullptr;
    unsigned* dsync = nullptr;
    BArgs args{};
    int rows = 2, threads = 256, blocks_per_sm = 1, grid = 0, sms = 0;
    double hist_bytes = 0.0;
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
    for (void* p : {(void*)b->dmem, (void*)b->ditems, (void*)b->dsync})
        if (p) cudaFree(p);
    delete b;
}

namespace tdc {
// a handle the persistent kernel can step: FP32, one wave, direct solve
static bool persistent_member(tdcfie_t h) {
    return h->plan && h->plan->prec == TDCFIE_FP32 && h->plan->R == 1 && !h->plan->gmres_on && h->plan->blocks;
}

template <int ROWS>
static cudaError_t launch_persistent_t(tdcfie_batch_t b, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->grid);
    cfg.blockDim = dim3(b->threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch_step<ROWS>, b->args);
}

static cudaError_t launch_persistent(tdcfie_batch_t b, cudaStream_t s) {
    switch (b->rows) {
        case 1: return launch_persistent_t<1>(b, s);
        case 4: return launch_persistent_t<4>(b, s);
        default: return launch_persistent_t<2>(b, s);
    }
}

static int max_blocks_per_sm(int rows, int threads) {
    int nb = 0;
    cudaError_t e;
    if (rows == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_step<1>, threads, 0);
    else if (rows == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_step<4>, threads, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_step<2>, threads, 0);
    return e == cudaSuccess ? nb : 0;
}

// work lists of the seven phases, longest items first (by the bytes they stream)
static cudaError_t build_persistent(tdcfie_batch_t b) {
    const int n = (int)b->hs.size();
    std::vector<BMember> mem(n);
    std::vector<std::vector<std::pair<double, BItem>>> lists(NPH);
    b->hist_bytes = 0.0;
    for (int s = 0; s < n; ++s) {
        tdcfie_t h = b->hs[s];
        StepPlan* p = h->plan;
        BMember& M = mem[s];
        M.ne = p->ne; M.nc = p->nc; M.nblk = p->nblk; M.ring = p->ring;
        M.blocks = (const float*)p->blocks; M.t0inv = (const float*)p->t0inv; M.pinv = (const float*)p->pinv;
        M.E = (float*)p->E; M.H = (float*)p->Hv; M.ringbuf = (float*)p->ringbuf;
        M.b = (float*)p->b; M.z = (float*)p->z; M.u = (float*)p->u; M.partial = (double*)p->partial;
        M.pptr = p->pptr; M.pnE = p->pnE; M.px = (const float*)p->px; M.pc = (const float*)p->pc;
        M.exc = h->dexc; M.m = h->dm; M.dt = h->dt; M.dtt = h->dtt; M.ctl = p->ctl;
        b->hist_bytes += (double)p->nblk * p->ne * p->ne * 4.0;
        for (int e = 0; e < p->ne; e += 32) {
            const BItem it{s, e, std::min(32, p->ne - e), 0};
            lists[PH_RHS].push_back({(double)p->ne, it});
            lists[PH_RED].push_back({(double)p->nblk, it});
            lists[PH_POUT].push_back({(double)p->ne, it});
        }
        for (int c = 0; c < p->nc; c += 32) lists[PH_PIN].push_back({(double)p->nc, BItem{s, c, std::min(32, p->nc - c), 0}});
        for (int r = 0; r < p->ne; r += BCH) {
            const int cnt = std::min(BCH, p->ne - r);
            for (int q = 0; q < p->nblk; q += BQ)
                lists[PH_HIST].push_back({(double)std::min(BQ, p->nblk - q) * p->ne * cnt, BItem{s, r, cnt, q}});
            lists[PH_SOLVE].push_back({(double)p->ne * cnt, BItem{s, r, cnt, 0}});
        }
        for (int r = 0; r < p->nc; r += BCH)
            lists[PH_PINV].push_back({(double)p->nc * std::min(BCH, p->nc - r), BItem{s, r, std::min(BCH, p->nc - r), 0}});
    }
    std::vector<BItem> all;
    std::vector<size_t> off(NPH);
    for (int ph = 0; ph < NPH; ++ph) {
        std::stable_sort(lists[ph].begin(), lists[ph].end(),
                         [](const std::pair<double, BItem>& x, const std::pair<double, BItem>& y) { return x.first > y.first; });
        off[ph] = all.size();
        for (auto& pr : lists[ph]) all.push_back(pr.second);
        b->args.nitems[ph] = (int)lists[ph].size();
    }
    cudaError_t e;
    if ((e = cudaMalloc(&b->dmem, sizeof(BMember) * n)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&b->ditems, sizeof(BItem) * all.size())) != cudaSuccess) return e;
    if ((e = cudaMalloc(&b->dsync, sizeof(unsigned) * (NPH + 3))) != cudaSuccess) return e;
    if ((e = cudaMemcpy(b->dmem, mem.data(), sizeof(BMember) * n, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(b->ditems, all.data(), sizeof(BItem) * all.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemset(b->dsync, 0, sizeof(unsigned) * (NPH + 3))) != cudaSuccess) return e;
    b->args.mem = b->dmem;
    b->args.nmem = n;
    for (int ph = 0; ph < NPH; ++ph) b->args.items[ph] = b->ditems + off[ph];
    b->args.sync = b->dsync;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    b->rows = 2;
    b->threads = 256;
    b->blocks_per_sm = std::max(1, std::min(2, max_blocks_per_sm(b->rows, b->threads)));
    b->grid = b->sms * b->blocks_per_sm;
    return cudaSuccess;
}
}  // namespace tdc

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
    b->persistent = true;
    for (int64_t i = 0; i < n; ++i) b->persistent = b->persistent && persistent_member(handles[i]);
    if (b->persistent) BK(build_persistent(b));
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
        e = cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaStreamBeginCapture");
        cudaError_t ce = cudaSuccess;
        if (b->persistent) {
            // one cooperative launch steps every member
            ce = launch_persistent(b, b->main);
            b->launches_per_step = 1;
        } else {
            // one step of every handle, each on its own branch of the graph
            ce = cudaEventRecord(b->fork, b->main);
            b->launches_per_step = 0;
            for (int64_t i = 0; i < n && ce == cudaSuccess; ++i) {
                ce = cudaStreamWaitEvent(b->branch[i], b->fork, 0);
                if (ce == cudaSuccess) ce = capture_step(b->hs[i], b->branch[i]);
                if (ce == cudaSuccess) ce = cudaEventRecord(b->joined[i], b->branch[i]);
                if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->main, b->joined[i], 0);
                b->launches_per_step += plan_launches_per_step(b->hs[i]);
            }
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
    if (b->persistent) {
        unsigned timeout = 0;
        e = cudaMemcpy(&timeout, b->dsync + NPH + 2, sizeof(unsigned), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch status");
        if (timeout) return fail(nullptr, TDCFIE_E_TIMEOUT, "a bounded grid-wide wait of the batch kernel ran out");
    }
    for (int64_t i = 0; i < n; ++i) {
        const tdcfie_status st = plan_check(b->hs[i]);
        if (st != TDCFIE_OK) return fail(nullptr, st, "batch handle " + std::to_string(i) + ": " + b->hs[i]->err);
    }
    return TDCFIE_OK;
}

extern "C" tdcfie_status tdcfie_batch_tune(tdcfie_batch_t b, int64_t steps_per_candidate, int32_t* config) {
    if (!b) return fail(nullptr, TDCFIE_E_ARG, "batch is NULL");
    if (steps_per_candidate < 1) return fail(nullptr, TDCFIE_E_ARG, "steps_per_candidate < 1");
    for (tdcfie_t h : b->hs)
        if (!h->excited || !h->plan)
            return fail(nullptr, TDCFIE_E_STATE, "set the excitation of every handle of the batch first");
    if (b->persistent) {
        cudaError_t e = cudaSetDevice(b->hs[0]->opts.device);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
        for (tdcfie_t h : b->hs) {
            const tdcfie_status st = plan_set_outputs(h, nullptr, nullptr);
            if (st != TDCFIE_OK) return st;
        }
        double best = 1e300;
        int br = b->rows, bt = b->threads, bb = b->blocks_per_sm;
        for (int rows : {1, 2, 4})
            for (int threads : {128, 256, 512}) {
                const int maxb = max_blocks_per_sm(rows, threads);
                for (int bps : {1, 2, 4}) {
                    if (bps > maxb) continue;
                    b->rows = rows; b->threads = threads; b->blocks_per_sm = bps; b->grid = b->sms * bps;
                    e = launch_persistent(b, b->main);                        // warm-up
                    if (e == cudaSuccess) e = cudaEventRecord(b->t0, b->main);
                    for (int64_t i = 0; i < steps_per_candidate && e == cudaSuccess; ++i) e = launch_persistent(b, b->main);
                    if (e == cudaSuccess) e = cudaEventRecord(b->t1, b->main);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(b->main);
                    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch autotuner");
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, b->t0, b->t1);
                    if (ms < best) { best = ms; br = rows; bt = threads; bb = bps; }
                }
            }
        b->rows = br; b->threads = bt; b->blocks_per_sm = bb; b->grid = b->sms * bb;
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
        unsigned timeout = 0;
        e = cudaMemcpy(&timeout, b->dsync + NPH + 2, sizeof(unsigned), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch status");
        if (timeout) return fail(nullptr, TDCFIE_E_TIMEOUT, "a bounded grid-wide wait of the batch kernel ran out");
        // the candidates marched the members: back to the start of the march
        for (tdcfie_t h : b->hs) {
            const tdcfie_status st = plan_reset(h);
            if (st != TDCFIE_OK) return st;
        }
    }
    if (config) {
        config[0] = b->persistent ? 1 : 0;
        config[1] = b->rows;
        config[2] = b->threads;
        config[3] = b->blocks_per_sm;
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
