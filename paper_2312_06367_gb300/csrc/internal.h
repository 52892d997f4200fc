// Internal declarations of the tdcfie library (product code; nothing here is shared with the
// oracle).  Natural units c = eta = 1.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tdcfie.h"

namespace tdc {

// ---------------------------------------------------------------- mesh and tables (host)
struct Mesh {
    int nv = 0, nc = 0, ne = 0, genus = 0;
    std::vector<double> V;        // nv x 3
    std::vector<int> F;           // nc x 3 (CCW about the outward normal)
    std::vector<int> E;           // ne x 2 (v-, v+), v- < v+, lexicographic order
    std::vector<int> cplus, cminus;
    std::vector<int> tedge;       // nc x 3: edge opposite local vertex j
    std::vector<double> tsign;    // nc x 3: +1 if the triangle is c+ of that edge
    std::vector<int> valence;     // nv: triangles at each vertex
    double D = 0.0;               // largest vertex-to-vertex distance
    // barycentric refinement
    int nf = 0;
    std::vector<double> fV;       // (nv + ne + nc) x 3
    std::vector<int> fF;          // nf x 3, coarse vertex first, CCW
    std::vector<int> fparent;     // nf: coarse triangle
    std::vector<int> fvert;       // nf: coarse vertex of the fine triangle
    std::vector<int> bc_ptr;      // nf + 1
    std::vector<int> bc_fn;       // BC function (edge) index
    std::vector<double> bc_phi;   // 3 outward fluxes per entry
};

// Returns "" on success, else the reason the mesh is rejected.
std::string build_mesh(const double* V, int64_t nv, const int32_t* F, int64_t nc, Mesh& m);

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n).
void gauss_legendre(int n, double* x, double* w);

// ---------------------------------------------------------------- quadrature rule constants
constexpr int NANG = 6;       // Gauss points per angular piece
constexpr int NRAD = 5;       // Gauss points per radial piece
constexpr double PIECE = 1.0; // largest psi / u width of a piece
constexpr int LAGW = 16;      // lag window held per thread in the retarded kernels

struct RuleTables {
    double ax[NANG], aw[NANG], rx[NRAD], rw[NRAD];
};

// ---------------------------------------------------------------- device assembly
struct DevMesh {
    const double* V; const int* F; const int* tedge; const double* tsign; const int* cplus_; const int* cminus_;
    const double* fV; const int* fF; const int* fparent; const int* fvert; const int* valence;
    const int* bc_ptr; const int* bc_fn; const double* bc_phi;
    int nv, nc, ne, nf;
};

void set_rule_tables(const RuleTables& r, cudaStream_t s);
// symmetric degree-5 rule on a triangle: per point barycentric (a, b, c) and weight (sum 1)
void triangle_rule7(double r7[7][4]);
void launch_retarded_efie(const DevMesh& m, double dt, int K, double T0, double D, double* S, double* Phi,
                          int order, cudaStream_t s);
void launch_retarded_mfie(const DevMesh& m, double dt, int K, double D, double* MM, int order, cudaStream_t s);
void launch_static(const DevMesh& m, double kappa, double* Zs, double* Psi, double* M, double* G, cudaStream_t s);

// ---------------------------------------------------------------- dense FP64 helpers (linalg.cu)
// C = alpha op(A) op(B) + beta C, row-major, FP64 (cuBLAS DGEMM).
void dgemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha, const double* A, int lda,
           const double* B, int ldb, double beta, double* C, int ldc);
void sgemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, float alpha, const float* A, int lda,
           const float* B, int ldb, float beta, float* C, int ldc);
// In-place inverse of an n x n row-major FP64 matrix (Gauss-Jordan, partial pivoting).
// Returns 0 on success, 1 if a zero pivot was met.
int invert(cudaStream_t s, double* A, int n, double* work);
void fill_identity(cudaStream_t s, double* A, int n, double scale);
void axpby(cudaStream_t s, int64_t n, double a, const double* x, double b, double* y);   // y = a x + b y
void scatter_incidence_dense(cudaStream_t s, const int* E2, int rows, int cols, double* out);   // +1/-1 rows
void cast_f64_f32(cudaStream_t s, const double* in, float* out, int64_t n);
void split_bf16(cudaStream_t s, const double* in, void* hi, void* lo, int64_t n);
void transpose(cudaStream_t s, const double* in, double* out, int rows, int cols);

// ---------------------------------------------------------------- hot path (march.cu)
struct StepPlan;   // defined in march.cu

struct Ctl {              // device-resident step state read by every kernel of a step
    int64_t n;            // current step (1-based)
    int64_t n0;           // step of the first output row of this tdcfie_step call
    void* out;            // currents_out of this call (nullptr: discard)
    int status;           // 0 ok, else a tdcfie_status recorded with bad_step
    int64_t bad_step;
    int timeout;          // set by a device-side bounded wait that ran out
    void* yout;           // optional y_n output of this call (nullptr: none)
    int noconv;           // set when a GMRES solve stopped above its tolerance (gmres_maxit reached)
    int64_t noconv_step;  // the first such step
};
}  // namespace tdc

struct tdcfie_s {
    tdcfie_opts opts;
    cudaStream_t stream = nullptr;
    bool own_stream = false;        // created by the library when opts.stream is NULL
    cudaEvent_t ev_in = nullptr;    // orders the library stream after the caller's legacy-stream work
    std::string err;
    tdc::Mesh mesh;
    double dt = 0, T0 = 0, dtt = 0, kappa = 0, alpha = 1;
    int64_t nt = 0;
    int K = 0;
    bool assembled = false, excited = false;
    bool formed_fp64 = false;   // T_k products formed in FP64 (opts.precision was FP64 at assembly)
    bool released = false;      // FP64 assembly matrices freed (tdcfie_release_assembly)
    // device mesh
    void* dmesh_buf = nullptr;
    tdc::DevMesh dm{};
    // FP64 assembled matrices (device)
    double *S = nullptr, *Phi = nullptr, *MM = nullptr, *Zs = nullptr, *Psi = nullptr, *Mst = nullptr, *G = nullptr;
    double *PS = nullptr, *L1 = nullptr, *L2 = nullptr, *A = nullptr, *T = nullptr, *T0inv = nullptr;
    double *H = nullptr, *Zh = nullptr;
    double *PinvS = nullptr;        // (Sigma^T Sigma)^+ (nc x nc)
    int *dE = nullptr, *dcp = nullptr, *dcm = nullptr, *dtedge = nullptr;
    double *dtsign = nullptr, *darea = nullptr;
    // path-precision blocks and march state
    tdc::StepPlan* plan = nullptr;
    // excitation
    int64_t R = 1;
    double* dexc = nullptr;   // R x 11: k(3), p(3), amp, t0, width, pad
    // timing
    double asm_s[6] = {0, 0, 0, 0, 0, 0};   // upload, retarded EFIE, retarded MFIE, static, formation, plan
    double last_step_ms = 0, last_hist_ms = 0, hist_bytes = 0;
    double step_bytes = 0;          // matrix bytes streamed per step by the whole plan
    int history_form = 0;           // tdcfie_history_form of the next plan
    int formulation = 0;            // tdcfie_formulation of the next plan
    int64_t last_launches = 0;
};

namespace tdc {
tdcfie_status fail(tdcfie_t h, tdcfie_status st, const std::string& msg);
tdcfie_status cuda_fail(tdcfie_t h, cudaError_t e, const char* where);
tdcfie_status build_plan(tdcfie_t h);
void free_plan(tdcfie_t h);
tdcfie_status plan_reset(tdcfie_t h);
tdcfie_status plan_step(tdcfie_t h, int64_t nsteps, void* out, void* yout = nullptr);
tdcfie_status plan_gmres_stats(tdcfie_t h, long long* out6);
tdcfie_status plan_set_solver(tdcfie_t h, int solver, int guess, double tol);
cudaError_t capture_step(tdcfie_t h, cudaStream_t s);
tdcfie_status plan_set_outputs(tdcfie_t h, void* out, void* yout);
tdcfie_status plan_check(tdcfie_t h);
int plan_launches_per_step(tdcfie_t h);
tdcfie_status far_field(tdcfie_t h, const void* currents, int64_t nt, double w, const double* rhat, int64_t ndir,
                        double* out);
}  // namespace tdc
