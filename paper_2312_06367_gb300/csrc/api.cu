// C ABI of the tdcfie library (include/tdcfie.h): argument checks, ownership, orchestration.
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>

#include "internal.h"
#include "plan.h"
#include "umma.h"

namespace tdc {
tdcfie_status form_operators(tdcfie_t h);

static thread_local std::string g_last_error;

tdcfie_status fail(tdcfie_t h, tdcfie_status st, const std::string& msg) {
    if (h) h->err = msg;
    g_last_error = msg;
    return st;
}
tdcfie_status cuda_fail(tdcfie_t h, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? TDCFIE_E_OOM : TDCFIE_E_CUDA, m);
}
}  // namespace tdc

using namespace tdc;

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return cuda_fail(h, e_, #x); } while (0)

extern "C" void tdcfie_default_opts(tdcfie_opts* o) {
    if (!o) return;
    o->precision = TDCFIE_FP64;
    o->solver = TDCFIE_SOLVE_DIRECT;
    o->gmres_tol = 1e-8;
    o->gmres_restart = 30;
    o->gmres_maxit = 300;
    o->guess = TDCFIE_GUESS_PREV;
    o->max_rhs = 1;
    o->stream = nullptr;
    o->device = 0;
    o->time_order = 1;
}

template <class T>
static cudaError_t put(tdcfie_t h, T** dst, const std::vector<T>& v) {
    cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * (v.size() ? v.size() : 1));
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, h->stream);
}

extern "C" tdcfie_status tdcfie_create(const double* vertices, int64_t nv, const int32_t* triangles, int64_t nc,
                                       double dt, int64_t nt, double alpha, const tdcfie_opts* opts, tdcfie_t* out) {
    if (!out) return fail(nullptr, TDCFIE_E_ARG, "out is NULL");
    *out = nullptr;
    if (!vertices || !triangles) return fail(nullptr, TDCFIE_E_ARG, "vertices/triangles is NULL");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(nullptr, TDCFIE_E_ARG, "dt must be positive and finite");
    if (nt < 0) return fail(nullptr, TDCFIE_E_ARG, "nt must be >= 0");
    if (!std::isfinite(alpha)) return fail(nullptr, TDCFIE_E_ARG, "alpha must be finite");
    tdcfie_opts o;
    tdcfie_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision < TDCFIE_FP64 || o.precision > TDCFIE_FP16X3) return fail(nullptr, TDCFIE_E_ARG, "bad precision");
    if (o.time_order != 1 && o.time_order != 2) return fail(nullptr, TDCFIE_E_ARG, "time_order must be 1 or 2");
    const bool tensor = o.precision == TDCFIE_BF16X3 || o.precision == TDCFIE_FP16X3;
    if (o.max_rhs < 1 || o.max_rhs > 4096) return fail(nullptr, TDCFIE_E_ARG, "max_rhs out of range [1, 4096]");
    if (tensor && o.max_rhs != 64)
        return fail(nullptr, TDCFIE_E_UNSUPPORTED, "the tensor-core paths march exactly 64 right-hand sides");
    if (!tensor && o.max_rhs > 8)
        return fail(nullptr, TDCFIE_E_UNSUPPORTED, "FP64/FP32 paths march at most 8 right-hand sides together");
    if (o.solver != TDCFIE_SOLVE_DIRECT && o.solver != TDCFIE_SOLVE_GMRES)
        return fail(nullptr, TDCFIE_E_ARG, "bad solver");
    if (o.solver == TDCFIE_SOLVE_GMRES && tensor)
        return fail(nullptr, TDCFIE_E_UNSUPPORTED, "GMRES runs on the FP64 and FP32 paths");
    if (o.solver == TDCFIE_SOLVE_GMRES && !(o.gmres_tol > 0.0 && o.gmres_tol < 1.0))
        return fail(nullptr, TDCFIE_E_ARG, "gmres_tol must be in (0, 1)");
    if (o.guess < TDCFIE_GUESS_ZERO || o.guess > TDCFIE_GUESS_MLP_EXTRAP) return fail(nullptr, TDCFIE_E_ARG, "bad guess");
    tdcfie_t h = new tdcfie_s();
    h->opts = o;
    h->R = o.max_rhs;
    h->stream = (cudaStream_t)o.stream;
    std::string why = build_mesh(vertices, nv, triangles, nc, h->mesh);
    if (!why.empty()) {
        delete h;
        return fail(nullptr, TDCFIE_E_MESH, why);
    }
    h->dt = dt;
    h->nt = nt;
    h->alpha = alpha;
    h->T0 = h->mesh.D;              // T0 = D / c
    h->dtt = dt / h->T0;            // Delta-tilde t
    h->kappa = 1.0 / dt;            // kappa = 1 / (c dt)
    h->K = (int)std::ceil(h->mesh.D / dt + h->opts.time_order + 1.0);   // q_0 reaches (order + 1) dt
    *out = h;
    return TDCFIE_OK;
}

// Upload the mesh tables on first use (create itself touches no device, so topology queries
// work without a GPU).
static tdcfie_status upload_mesh(tdcfie_t h) {
    if (h->dm.V) return TDCFIE_OK;
    cudaError_t e = cudaSetDevice(h->opts.device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if (!h->stream) {
        // a graph cannot be captured on the legacy default stream: use a stream of our own
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamCreate");
        h->own_stream = true;
    }
    e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventCreate");
    const Mesh& M = h->mesh;
    DevMesh& d = h->dm;
    double *V, *tsign, *fV, *bc_phi;
    int *F, *tedge, *cp, *cm, *fF, *fparent, *fvert, *val, *bc_ptr, *bc_fn;
    if ((e = put(h, &V, M.V)) || (e = put(h, &F, M.F)) || (e = put(h, &tedge, M.tedge)) || (e = put(h, &tsign, M.tsign)) ||
        (e = put(h, &cp, M.cplus)) || (e = put(h, &cm, M.cminus)) || (e = put(h, &fV, M.fV)) || (e = put(h, &fF, M.fF)) ||
        (e = put(h, &fparent, M.fparent)) || (e = put(h, &fvert, M.fvert)) || (e = put(h, &val, M.valence)) ||
        (e = put(h, &bc_ptr, M.bc_ptr)) || (e = put(h, &bc_fn, M.bc_fn)) || (e = put(h, &bc_phi, M.bc_phi)))
        return cuda_fail(h, e, "upload mesh");
    d.V = V; d.F = F; d.tedge = tedge; d.tsign = tsign; d.cplus_ = cp; d.cminus_ = cm;
    d.fV = fV; d.fF = fF; d.fparent = fparent; d.fvert = fvert; d.valence = val;
    d.bc_ptr = bc_ptr; d.bc_fn = bc_fn; d.bc_phi = bc_phi;
    d.nv = M.nv; d.nc = M.nc; d.ne = M.ne; d.nf = M.nf;
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "upload mesh");
    return TDCFIE_OK;
}

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

extern "C" tdcfie_status tdcfie_assemble(tdcfie_t h) {
    if (!h) return fail(nullptr, TDCFIE_E_ARG, "handle is NULL");
    double t0 = now_s();
    {
        tdcfie_status st0 = upload_mesh(h);
        if (st0 != TDCFIE_OK) return st0;
    }
    h->asm_s[0] = now_s() - t0;
    const Mesh& M = h->mesh;
    cudaStream_t s = h->stream;
    const int64_t ne = M.ne, nc = M.nc, nv = M.nv, K = h->K;
    RuleTables rt;
    gauss_legendre(NANG, rt.ax, rt.aw);
    gauss_legendre(NRAD, rt.rx, rt.rw);
    set_rule_tables(rt, s);
    auto zalloc = [&](double** p, int64_t n) -> cudaError_t {
        if (*p) return cudaMemsetAsync(*p, 0, sizeof(double) * n, s);
        cudaError_t e = cudaMalloc((void**)p, sizeof(double) * n);
        if (e != cudaSuccess) return e;
        return cudaMemsetAsync(*p, 0, sizeof(double) * n, s);
    };
    CK(zalloc(&h->S, K * ne * ne));
    CK(zalloc(&h->Phi, K * nc * nc));
    CK(zalloc(&h->MM, K * ne * ne));
    CK(zalloc(&h->Zs, ne * ne));
    CK(zalloc(&h->Psi, nv * nv));
    CK(zalloc(&h->Mst, ne * ne));
    CK(zalloc(&h->G, ne * ne));
    CK(cudaStreamSynchronize(s));
    t0 = now_s();
    launch_retarded_efie(h->dm, h->dt, h->K, h->T0, M.D, h->S, h->Phi, h->opts.time_order, s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    h->asm_s[1] = now_s() - t0;
    t0 = now_s();
    launch_retarded_mfie(h->dm, h->dt, h->K, M.D, h->MM, h->opts.time_order, s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    h->asm_s[2] = now_s() - t0;
    t0 = now_s();
    launch_static(h->dm, h->kappa, h->Zs, h->Psi, h->Mst, h->G, s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    h->asm_s[3] = now_s() - t0;
    t0 = now_s();
    tdcfie_status st = form_operators(h);
    if (st != TDCFIE_OK) return st;
    h->asm_s[4] = now_s() - t0;
    h->assembled = true;
    h->formed_fp64 = h->opts.precision == TDCFIE_FP64;
    t0 = now_s();
    st = build_plan(h);
    if (st != TDCFIE_OK) return st;
    h->asm_s[5] = now_s() - t0;
    return TDCFIE_OK;
}

extern "C" tdcfie_status tdcfie_set_excitation(tdcfie_t h, const tdcfie_plane_waves* exc) {
    if (!h || !exc) return fail(h, TDCFIE_E_ARG, "NULL argument");
    if (!h->assembled) return fail(h, TDCFIE_E_STATE, "call tdcfie_assemble first");
    if (exc->R != h->R) return fail(h, TDCFIE_E_ARG, "excitation R differs from opts.max_rhs");
    if (!exc->k_hat || !exc->pol || !exc->amp || !exc->t0 || !exc->width) return fail(h, TDCFIE_E_ARG, "NULL array");
    std::vector<double> buf(11 * h->R, 0.0);
    for (int64_t r = 0; r < h->R; ++r) {
        for (int i = 0; i < 3; ++i) { buf[11 * r + i] = exc->k_hat[3 * r + i]; buf[11 * r + 3 + i] = exc->pol[3 * r + i]; }
        buf[11 * r + 6] = exc->amp[r];
        buf[11 * r + 7] = exc->t0[r];
        buf[11 * r + 8] = exc->width[r];
        if (!(exc->width[r] > 0.0)) return fail(h, TDCFIE_E_ARG, "width must be positive");
        for (int i = 0; i < 9; ++i) if (!std::isfinite(buf[11 * r + i])) return fail(h, TDCFIE_E_ARG, "non-finite excitation");
    }
    if (!h->dexc) CK(cudaMalloc(&h->dexc, sizeof(double) * buf.size()));
    CK(cudaMemcpyAsync(h->dexc, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice, h->stream));
    h->excited = true;
    return plan_reset(h);
}

extern "C" tdcfie_status tdcfie_step(tdcfie_t h, int64_t nsteps, void* out) {
    if (!h) return fail(nullptr, TDCFIE_E_ARG, "handle is NULL");
    if (!h->excited) return fail(h, TDCFIE_E_STATE, "call tdcfie_set_excitation first");
    if (nsteps < 0) return fail(h, TDCFIE_E_ARG, "nsteps < 0");
    if (nsteps == 0) return TDCFIE_OK;
    return plan_step(h, nsteps, out);
}

extern "C" tdcfie_status tdcfie_step_y(tdcfie_t h, int64_t nsteps, void* currents_out, void* y_out) {
    if (!h) return fail(nullptr, TDCFIE_E_ARG, "handle is NULL");
    if (!h->excited) return fail(h, TDCFIE_E_STATE, "call tdcfie_set_excitation first");
    if (nsteps < 0) return fail(h, TDCFIE_E_ARG, "nsteps < 0");
    if (h->opts.precision == TDCFIE_BF16X3 || h->opts.precision == TDCFIE_FP16X3)
        return fail(h, TDCFIE_E_UNSUPPORTED, "y output is built for the FP64 and FP32 paths");
    if (nsteps == 0) return TDCFIE_OK;
    return plan_step(h, nsteps, currents_out, y_out);
}

extern "C" tdcfie_status tdcfie_gmres_stats(tdcfie_t h, int64_t* inner_iterations, int64_t* steps,
                                            int64_t* max_per_step, int64_t* not_converged) {
    if (!h) return fail(nullptr, TDCFIE_E_ARG, "handle is NULL");
    long long v[6] = {0, 0, 0, 0, 0, 0};
    tdcfie_status st = plan_gmres_stats(h, v);
    if (st != TDCFIE_OK) return st;
    if (inner_iterations) *inner_iterations = v[0];
    if (steps) *steps = v[1];
    if (max_per_step) *max_per_step = v[2];
    if (not_converged) *not_converged = v[4];
    return TDCFIE_OK;
}

extern "C" tdcfie_status tdcfie_replan(tdcfie_t h, int precision, int64_t max_rhs) {
    if (!h) return fail(nullptr, TDCFIE_E_ARG, "handle is NULL");
    if (!h->assembled) return fail(h, TDCFIE_E_STATE, "call tdcfie_assemble first");
    if (precision < TDCFIE_FP64 || precision > TDCFIE_FP16X3) return fail(h, TDCFIE_E_ARG, "bad precision");
    const bool tensor = precision == TDCFIE_BF16X3 || precision == TDCFIE_FP16X3;
    if (max_rhs < 1 || (tensor && max_rhs != 64) || (!tensor && max_rhs > 8))
        return fail(h, TDCFIE_E_UNSUPPORTED, "R must be 64 on the tensor-core paths and 1..8 on FP64/FP32");
    if (precision == TDCFIE_FP64 && !h->formed_fp64)
        return fail(h, TDCFIE_E_UNSUPPORTED, "the FP64 path needs blocks formed in FP64 (assemble with precision FP64)");
    if (h->released) return fail(h, TDCFIE_E_STATE, "the FP64 assembly was released (tdcfie_release_assembly)");
    if (tensor && h->formulation != TDCFIE_FORMULATION_QHP_CFIE)
        return fail(h, TDCFIE_E_UNSUPPORTED, "the comparison formulation runs on the dense FP64 and FP32 paths");
    if (tensor && h->opts.solver == TDCFIE_SOLVE_GMRES) h->opts.solver = TDCFIE_SOLVE_DIRECT;
    h->opts.precision = precision;
    h->opts.max_rhs = max_rhs;
    if (h->R != max_rhs && h->dexc) {
        cudaFree(h->dexc);
        h->dexc = nullptr;
    }
    h->R = max_rhs;
    h->excited = false;
    return build_plan(h);
}

extern "C" tdcfie_status tdcfie_set_solver(tdcfie_t h, int solver, int guess, double gmres_tol) {
    if (!h) return fail(nullptr, TDCFIE_E_ARG, "handle is NULL");
    if (!h->assembled || !h->plan) return fail(h, TDCFIE_E_STATE, "call tdcfie_assemble first");
    if (solver != TDCFIE_SOLVE_DIRECT && solver != TDCFIE_SOLVE_GMRES) return fail(h, TDCFIE_E_ARG, "bad solver");
    if (guess < TDCFIE_GUESS_ZERO || guess > TDCFIE_GUESS_MLP_EXTRAP) return fail(h, TDCFIE_E_ARG, "bad guess");
    if (solver == TDCFIE_SOLVE_GMRES && !(gmres_tol > 0.0 && gmres_tol < 1.0))
        return fail(h, TDCFIE_E_ARG, "gmres_tol must be in (0, 1)");
    if (solver == TDCFIE_SOLVE_GMRES && h->released && !h->plan->t0mat)
        return fail(h, TDCFIE_E_STATE, "the FP64 assembly was released (tdcfie_release_assembly)");
    return plan_set_solver(h, solver, guess, gmres_tol);
}

extern "C" tdcfie_status tdcfie_set_history_form(tdcfie_t h, int form) {
    if (!h) return fail(nullptr, TDCFIE_E_ARG, "handle is NULL");
    if (form != TDCFIE_HISTORY_DENSE && form != TDCFIE_HISTORY_FACTORED) return fail(h, TDCFIE_E_ARG, "bad history form");
    if (!h->assembled || !h->plan) return fail(h, TDCFIE_E_STATE, "call tdcfie_assemble first");
    if (form == TDCFIE_HISTORY_FACTORED) {
        if (h->opts.precision != TDCFIE_FP64 && h->opts.precision != TDCFIE_FP32)
            return fail(h, TDCFIE_E_UNSUPPORTED, "the factored history form runs on the FP64 and FP32 paths");
        if (h->opts.solver != TDCFIE_SOLVE_DIRECT)
            return fail(h, TDCFIE_E_UNSUPPORTED, "the factored history form uses the direct solve");
        if (h->formulation != TDCFIE_FORMULATION_QHP_CFIE)
            return fail(h, TDCFIE_E_UNSUPPORTED, "the comparison formulation runs on the dense FP64 and FP32 paths");
    }
    if (h->released) return fail(h, TDCFIE_E_STATE, "the FP64 assembly was released (tdcfie_release_assembly)");
    const int old = h->history_form;
    h->history_form = form;
    h->excited = false;
    const tdcfie_status st = build_plan(h);
    if (st != TDCFIE_OK) {
        h->history_form = old;
        free_plan(h);
    }
    return st;
}

extern "C" tdcfie_status tdcfie_set_formulation(tdcfie_t h, int formulation) {
    if (!h) return fail(nullptr, TDCFIE_E_ARG, "handle is NULL");
    if (formulation != TDCFIE_FORMULATION_QHP_CFIE && formulation != TDCFIE_FORMULATION_MFIE)
        return fail(h, TDCFIE_E_ARG, "bad formulation");
    if (!h->assembled || !h->plan) return fail(h, TDCFIE_E_STATE, "call tdcfie_assemble first");
    if (formulation != TDCFIE_FORMULATION_QHP_CFIE) {
        if (h->opts.precision != TDCFIE_FP64 && h->opts.precision != TDCFIE_FP32)
            return fail(h, TDCFIE_E_UNSUPPORTED, "the comparison formulation runs on the dense FP64 and FP32 paths");
        if (h->opts.solver != TDCFIE_SOLVE_DIRECT)
            return fail(h, TDCFIE_E_UNSUPPORTED, "the comparison formulation uses the direct solve");
        if (h->history_form != TDCFIE_HISTORY_DENSE)
            return fail(h, TDCFIE_E_UNSUPPORTED, "the comparison formulation runs on the dense FP64 and FP32 paths");
    }
    if (h->released) return fail(h, TDCFIE_E_STATE, "the FP64 assembly was released (tdcfie_release_assembly)");
    const int old = h->formulation;
    h->formulation = formulation;
    h->excited = false;
    const tdcfie_status st = build_plan(h);
    if (st != TDCFIE_OK) {
        h->formulation = old;
        free_plan(h);
    }
    return st;
}

extern "C" tdcfie_status tdcfie_history_stats(tdcfie_t h, int32_t* form, int64_t* nnz, double* history_bytes,
                                              double* step_bytes) {
    if (!h) return fail(nullptr, TDCFIE_E_ARG, "handle is NULL");
    if (!h->plan) return fail(h, TDCFIE_E_STATE, "call tdcfie_assemble first");
    if (form) *form = h->plan->fact ? TDCFIE_HISTORY_FACTORED : TDCFIE_HISTORY_DENSE;
    if (nnz) *nnz = h->plan->fact ? fact_nnz(h->plan, false) : 0;
    if (history_bytes) *history_bytes = h->hist_bytes;
    if (step_bytes) *step_bytes = h->step_bytes;
    return TDCFIE_OK;
}

extern "C" tdcfie_status tdcfie_far_field(tdcfie_t h, const void* currents, int64_t nt, double w, const double* rhat,
                                          int64_t ndir, double* out) {
    if (!h) return fail(nullptr, TDCFIE_E_ARG, "handle is NULL");
    if (!h->assembled || !h->plan) return fail(h, TDCFIE_E_STATE, "call tdcfie_assemble first");
    if (!currents || !rhat || !out || nt < 1 || ndir < 1 || !(w >= 0.0) || !std::isfinite(w))
        return fail(h, TDCFIE_E_ARG, "far field: NULL buffer, nt < 1, ndir < 1 or a bad frequency");
    if (ndir > 65535) return fail(h, TDCFIE_E_ARG, "far field: at most 65535 directions per call");
    for (int64_t d = 0; d < ndir; ++d) {
        const double n2 = rhat[3 * d] * rhat[3 * d] + rhat[3 * d + 1] * rhat[3 * d + 1] + rhat[3 * d + 2] * rhat[3 * d + 2];
        if (!(std::fabs(n2 - 1.0) < 1e-9)) return fail(h, TDCFIE_E_ARG, "far field: directions must be unit vectors");
    }
    return far_field(h, currents, nt, w, rhat, ndir, out);
}

extern "C" tdcfie_status tdcfie_march(tdcfie_t h, const tdcfie_plane_waves* exc, void* out, int out_on_host) {
    tdcfie_status st = tdcfie_set_excitation(h, exc);
    if (st != TDCFIE_OK) return st;
    if (!out_on_host) return tdcfie_step(h, h->nt, out);
    const size_t es = h->opts.precision == TDCFIE_FP64 ? 8 : 4;
    const size_t bytes = es * (size_t)h->nt * h->R * h->mesh.ne;
    void* d = nullptr;
    if (out) CK(cudaMalloc(&d, bytes ? bytes : 1));
    st = tdcfie_step(h, h->nt, d);
    if (st == TDCFIE_OK && out) {
        cudaError_t e = cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) st = cuda_fail(h, e, "copy currents to host");
    }
    if (d) cudaFree(d);
    return st;
}

extern "C" tdcfie_status tdcfie_info(tdcfie_t h, int64_t* ne, int64_t* nc, int64_t* nv, int64_t* K, int32_t* genus,
                                     double* D) {
    if (!h) return fail(nullptr, TDCFIE_E_ARG, "handle is NULL");
    if (ne) *ne = h->mesh.ne;
    if (nc) *nc = h->mesh.nc;
    if (nv) *nv = h->mesh.nv;
    if (K) *K = h->K;
    if (genus) *genus = h->mesh.genus;
    if (D) *D = h->mesh.D;
    return TDCFIE_OK;
}

extern "C" tdcfie_status tdcfie_topology(tdcfie_t h, int32_t* edges, int32_t* cplus, int32_t* cminus) {
    if (!h) return fail(nullptr, TDCFIE_E_ARG, "handle is NULL");
    const Mesh& M = h->mesh;
    if (edges) std::memcpy(edges, M.E.data(), sizeof(int) * M.E.size());
    if (cplus) std::memcpy(cplus, M.cplus.data(), sizeof(int) * M.ne);
    if (cminus) std::memcpy(cminus, M.cminus.data(), sizeof(int) * M.ne);
    return TDCFIE_OK;
}

extern "C" tdcfie_status tdcfie_bc_table(tdcfie_t h, int64_t* nentries, int32_t* fine_tri, int32_t* fn,
                                         double* phi, double* fine_vertices, int32_t* fine_triangles) {
    if (!h) return fail(nullptr, TDCFIE_E_ARG, "handle is NULL");
    const Mesh& M = h->mesh;
    if (nentries) *nentries = (int64_t)M.bc_fn.size();
    if (fine_tri)
        for (int t = 0; t < M.nf; ++t)
            for (int e = M.bc_ptr[t]; e < M.bc_ptr[t + 1]; ++e) fine_tri[e] = t;
    if (fn) std::memcpy(fn, M.bc_fn.data(), sizeof(int) * M.bc_fn.size());
    if (phi) std::memcpy(phi, M.bc_phi.data(), sizeof(double) * M.bc_phi.size());
    if (fine_vertices) std::memcpy(fine_vertices, M.fV.data(), sizeof(double) * M.fV.size());
    if (fine_triangles) std::memcpy(fine_triangles, M.fF.data(), sizeof(int) * M.fF.size());
    return TDCFIE_OK;
}

extern "C" tdcfie_status tdcfie_get_matrix(tdcfie_t h, int which, int64_t k, double* host_out) {
    if (!h || !host_out) return fail(h, TDCFIE_E_ARG, "NULL argument");
    if (!h->assembled) return fail(h, TDCFIE_E_STATE, "not assembled");
    if (h->released) return fail(h, TDCFIE_E_STATE, "the FP64 assembly was released (tdcfie_release_assembly)");
    const int64_t ne = h->mesh.ne, NN = ne * ne;
    const double* src = nullptr;
    const bool lagged = (which >= 0 && which <= 3) || which == 11;
    if (lagged && (k < 0 || k >= h->K)) return fail(h, TDCFIE_E_ARG, "lag out of range");
    switch (which) {
        case 0: src = h->T + k * NN; break;
        case 1: src = h->S + k * NN; break;
        case 3: src = h->MM + k * NN; break;
        case 4: src = h->G; break;
        case 5: src = h->Zs; break;
        case 6: src = h->Zh; break;
        case 7: src = h->Mst; break;
        case 8: src = h->PS; break;
        case 9: src = h->L1; break;
        case 10: src = h->L2; break;
        case 11:
            CK(cudaMemcpy(host_out, h->Phi + k * h->mesh.nc * h->mesh.nc, sizeof(double) * h->mesh.nc * h->mesh.nc,
                          cudaMemcpyDeviceToHost));
            return TDCFIE_OK;
        case 2: {
            // H_k = Sigma Phi_k Sigma^T, expanded on the host
            const Mesh& M = h->mesh;
            const int64_t nc = M.nc;
            std::vector<double> phi(nc * nc);
            CK(cudaMemcpy(phi.data(), h->Phi + k * nc * nc, sizeof(double) * nc * nc, cudaMemcpyDeviceToHost));
            for (int64_t a = 0; a < ne; ++a)
                for (int64_t b = 0; b < ne; ++b) {
                    const int ap = M.cplus[a], am = M.cminus[a], bp = M.cplus[b], bm = M.cminus[b];
                    host_out[a * ne + b] = phi[ap * nc + bp] - phi[ap * nc + bm] - phi[am * nc + bp] + phi[am * nc + bm];
                }
            return TDCFIE_OK;
        }
        default: return fail(h, TDCFIE_E_ARG, "unknown matrix id");
    }
    CK(cudaMemcpy(host_out, src, sizeof(double) * NN, cudaMemcpyDeviceToHost));
    return TDCFIE_OK;
}

extern "C" tdcfie_status tdcfie_last_timing(tdcfie_t h, double* step_ms, double* history_ms, double* history_bytes,
                                            int64_t* launches) {
    if (!h) return fail(nullptr, TDCFIE_E_ARG, "handle is NULL");
    if (step_ms) *step_ms = h->last_step_ms;
    if (history_ms) *history_ms = h->last_hist_ms;
    if (history_bytes) *history_bytes = h->hist_bytes;
    if (launches) *launches = h->last_launches;
    return TDCFIE_OK;
}

extern "C" tdcfie_status tdcfie_assembly_timing(tdcfie_t h, double* seconds) {
    if (!h || !seconds) return fail(h, TDCFIE_E_ARG, "NULL argument");
    for (int i = 0; i < 6; ++i) seconds[i] = h->asm_s[i];
    return TDCFIE_OK;
}

extern "C" tdcfie_status tdcfie_release_assembly(tdcfie_t h) {
    if (!h) return fail(nullptr, TDCFIE_E_ARG, "handle is NULL");
    if (!h->assembled || !h->plan) return fail(h, TDCFIE_E_STATE, "call tdcfie_assemble first");
    CK(cudaStreamSynchronize(h->stream));
    double** ptrs[] = {&h->S, &h->Phi, &h->MM, &h->Zs, &h->Psi, &h->Mst, &h->G, &h->PS, &h->L1, &h->L2, &h->A, &h->T,
                       &h->T0inv, &h->H, &h->Zh};
    for (double** q : ptrs)
        if (*q) {
            CK(cudaFree(*q));
            *q = nullptr;
        }
    h->released = true;
    return TDCFIE_OK;
}

extern "C" tdcfie_status tdcfie_destroy(tdcfie_t h) {
    if (!h) return TDCFIE_OK;
    free_plan(h);
    const void* ptrs[] = {h->dm.V, h->dm.F, h->dm.tedge, h->dm.tsign, h->dm.cplus_, h->dm.cminus_, h->dm.fV, h->dm.fF,
                          h->dm.fparent, h->dm.fvert, h->dm.valence, h->dm.bc_ptr, h->dm.bc_fn, h->dm.bc_phi,
                          h->S, h->Phi, h->MM, h->Zs, h->Psi, h->Mst, h->G, h->PS, h->L1, h->L2, h->A, h->T, h->T0inv,
                          h->H, h->Zh, h->PinvS, h->dexc};
    for (const void* p : ptrs) if (p) cudaFree(const_cast<void*>(p));
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return TDCFIE_OK;
}

extern "C" const char* tdcfie_last_error(tdcfie_t h) {
    if (h) return h->err.c_str();
    return g_last_error.c_str();
}

extern "C" tdcfie_status tdcfie_tc_gemm(int precision, const double* blocks, int64_t nblk, int64_t rows, int64_t cols,
                                        const double* x, int64_t R, double* out, void* stream) {
    return tc_gemm(precision, blocks, nblk, rows, cols, x, R, out, (cudaStream_t)stream);
}
