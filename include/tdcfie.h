/*
 * tdcfie.h -- C ABI of the GB300 (sm_103a) marching-on-in-time solver for the quasi-Helmholtz
 * projected, Yukawa-Calderon preconditioned time-domain combined field integral equation
 * (Le, Cordel, Andriulli, Cools, "A Stabilized Time-Domain Combined Field Integral Equation Using
 * the Quasi-Helmholtz Projectors", arXiv 2312.06367).
 *
 * Natural units: c = eta = 1 (so kappa = 1/dt and T0 = D).  All entry points return a
 * tdcfie_status (0 = success, negative = error) and never abort; tdcfie_last_error() gives a
 * one-line message.  Handles are not thread-safe; every device operation of a handle runs on
 * opts.stream.  Host arrays passed in are copied; device arrays passed in are used in place and
 * remain owned by the caller.
 */
#ifndef TDCFIE_H
#define TDCFIE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdcfie_s* tdcfie_t;

typedef enum {
    TDCFIE_OK = 0,
    TDCFIE_E_ARG = -1,         /* invalid argument (null pointer, size <= 0, dt <= 0, ...) */
    TDCFIE_E_MESH = -2,        /* mesh not closed / not manifold / inconsistently oriented / disconnected */
    TDCFIE_E_OOM = -3,         /* device or host allocation failed */
    TDCFIE_E_CUDA = -4,        /* a CUDA runtime call failed (message holds the CUDA error string) */
    TDCFIE_E_NOCONV = -5,      /* GMRES did not reach the tolerance (step index in the message) */
    TDCFIE_E_TIMEOUT = -6,     /* a bounded device-side wait ran out */
    TDCFIE_E_NONFINITE = -7,   /* a NaN/Inf was produced (step index in the message) */
    TDCFIE_E_STATE = -8,       /* call out of order (e.g. march before assemble) */
    TDCFIE_E_UNSUPPORTED = -9  /* option combination not built (e.g. BF16X3 with R not a multiple of 16) */
} tdcfie_status;

/* Arithmetic of the per-step history sum and solve (Sec. IV-B).  FP64: everything FP64.
 * FP32: FP32 matrices and vectors on CUDA cores; every row dot product is accumulated error-free
 * (FMA product errors and TwoSum) and combined in FP64.  BF16X3: matrices and vectors
 * split into bf16 hi + lo, three tensor-core products (hi*hi + hi*lo + lo*hi) with FP32
 * accumulation.  FP16X3: the same with fp16 halves of power-of-two scaled values (per-row scales
 * of every matrix block, one scale per vector slot and right-hand side), about 2^-22 instead of
 * 2^-16 relative per stored entry at the same 4 bytes per entry.  BF16X3 and FP16X3 march exactly
 * 64 right-hand sides; FP64 and FP32 at most 8. */
typedef enum { TDCFIE_FP64 = 0, TDCFIE_FP32 = 1, TDCFIE_BF16X3 = 2, TDCFIE_FP16X3 = 3 } tdcfie_precision;
/* Solve with T_0 each step: DIRECT = explicit FP64-factored inverse applied in path precision;
 * GMRES = restarted GMRES on T_0: inner Arnoldi cycles of gmres_restart iterations with the
 * path-precision T_0 and CGS2 orthogonalisation in FP64, outer cycles restart from the true FP64
 * residual until ||b - T_0 y|| <= gmres_tol ||b|| (at most gmres_maxit inner iterations in all).
 * Initial guess: ZERO, PREV (y_{n-1}), EXTRAP (cubic extrapolation of y_{n-1..n-4}), or a learned
 * guess (MLP on top of y_{n-1}, MLP_EXTRAP on top of the extrapolation; see tdcfie_mlp_*); y_i = 0
 * for i <= 0.  FP64 and FP32 paths. */
typedef enum { TDCFIE_SOLVE_DIRECT = 0, TDCFIE_SOLVE_GMRES = 1 } tdcfie_solver;
typedef enum {
    TDCFIE_GUESS_ZERO = 0,       /* x0 = 0 */
    TDCFIE_GUESS_PREV = 1,       /* x0 = y_{n-1} */
    TDCFIE_GUESS_MLP = 2,        /* x0 = y_{n-1} + s f(x): the learned increment */
    TDCFIE_GUESS_EXTRAP = 3,     /* x0 = 4 y_{n-1} - 6 y_{n-2} + 4 y_{n-3} - y_{n-4}: cubic extrapolation */
    TDCFIE_GUESS_MLP_EXTRAP = 4  /* x0 = cubic extrapolation + s f(x): the learned correction to it */
} tdcfie_guess;

typedef struct {
    int precision;        /* tdcfie_precision, default TDCFIE_FP64 */
    int solver;           /* tdcfie_solver, default TDCFIE_SOLVE_DIRECT */
    double gmres_tol;     /* relative FP64 residual target, default 1e-8 */
    int gmres_restart;    /* Krylov dimension per cycle, default 30 */
    int gmres_maxit;      /* total iteration cap per step, default 300 */
    int guess;            /* tdcfie_guess for GMRES, default TDCFIE_GUESS_PREV */
    int64_t max_rhs;      /* R: right-hand sides (incident waves) marched together, default 1 */
    void* stream;         /* cudaStream_t; NULL = the legacy default stream */
    int device;           /* CUDA device ordinal, default 0 */
    int time_order;       /* temporal basis: 1 (default) the hat h_i with the C1 quadratic q_i of
                             Sec. IV-A; 2 the shifted quadratic Lagrange h_i with the q_i of the
                             remark closing Sec. IV-B (q_i' = (h_i - h_{i+1})/dt), K one larger */
} tdcfie_opts;

/* Fill *opts with the defaults above. */
void tdcfie_default_opts(tdcfie_opts* opts);

/*
 * Create a solver for the closed, connected, orientable triangulated surface Gamma (Sec. II-A):
 *   vertices  host, nv x 3 float64, row-major;
 *   triangles host, nc x 3 int32 vertex indices, counter-clockwise about the outward normal.
 * dt: time step (> 0); nt: steps a march produces; alpha: coupling of the MFIE part (the
 * paper's eta^2 in Eq. qHP_TDCFIE; 1 in natural units).
 * Builds the edge table (edges = sorted unique vertex pairs, oriented min -> max), the
 * incidence matrices Lambda and Sigma (Sec. II-D), the barycentric refinement and the BC table
 * (Sec. II-C), D (largest vertex distance), T0 = D, and the number of time blocks
 * K = ceil(D/dt + time_order + 1).  Host work only (no device is touched until tdcfie_assemble, which
 * uploads the tables).  *out receives the handle.
 * Errors: TDCFIE_E_ARG, TDCFIE_E_MESH, TDCFIE_E_OOM, TDCFIE_E_CUDA.
 */
tdcfie_status tdcfie_create(const double* vertices, int64_t nv, const int32_t* triangles, int64_t nc,
                            double dt, int64_t nt, double alpha, const tdcfie_opts* opts, tdcfie_t* out);

/*
 * Assemble on the device (FP64): retarded matrices S_k, H_k, MM_k (Sec. II-C, IV-A), the static
 * Yukawa matrices Z^s, Z^h, M and the Gram matrix G (Sec. II-B, II-C), the projectors
 * (Sec. II-D), L1 = Z~ G^-T and L2 = X~ G^-1 (Sec. III), the dense blocks
 * T_k = L1 ZZ~_k + alpha L2 XX~_k of Eq. dis_TD_CFIE, the inverse of T_0, and their copies in
 * the path precision.  One-time; not part of a step.
 */
tdcfie_status tdcfie_assemble(tdcfie_t h);

/* Plane waves e_in = amp p exp(-((t - k.r - t0)/width)^2), h_in = k x e_in (Sec. V, natural
 * units).  Host arrays: k_hat R x 3 (unit), pol R x 3 (unit, orthogonal to k), amp, t0, width R. */
typedef struct {
    int64_t R;
    const double* k_hat;
    const double* pol;
    const double* amp;
    const double* t0;
    const double* width;
} tdcfie_plane_waves;

/* Copy the excitation to the device (R must equal opts.max_rhs) and reset the march to n = 0
 * (history cleared: y_i = 0 for i <= 0, causality of Sec. II-A). */
tdcfie_status tdcfie_set_excitation(tdcfie_t h, const tdcfie_plane_waves* exc);

/*
 * Advance the march by nsteps steps of the MOT recurrence (Sec. IV-B):
 *   r_n = -L1 (dtt P^LH + P^S) e(t_n) + alpha L2 h(t_n)
 *   y_n = T_0^-1 (r_n - sum_{k=1}^{K-1} T_k y_{n-k})
 *   j_n = P^LH y_n + P^S (y_n - y_{n-1}) / dtt          (Eq. post_processing)
 * currents_out: DEVICE buffer of nsteps x R x N_E elements (step-major, then incident wave, then
 * edge), float64 for TDCFIE_FP64 and float32 otherwise; may be NULL to discard the currents.
 * The march state (step counter, ring of the last K-1 y, the last y) persists across calls.
 */
tdcfie_status tdcfie_step(tdcfie_t h, int64_t nsteps, void* currents_out);

/* tdcfie_step that also writes the auxiliary unknown y_n (Eq. y_expansion coefficients) of every
 * step to y_out (DEVICE, nsteps x R x N_E, path dtype; NULL = none).  FP64 and FP32 paths. */
tdcfie_status tdcfie_step_y(tdcfie_t h, int64_t nsteps, void* currents_out, void* y_out);

/* GMRES statistics since the last set_excitation (opts.solver = TDCFIE_SOLVE_GMRES): total inner
 * iterations over all steps and right-hand sides, steps solved, the largest per-step count, and the
 * number of (step, right-hand side) solves left above gmres_tol after the last outer cycle. */
tdcfie_status tdcfie_gmres_stats(tdcfie_t h, int64_t* inner_iterations, int64_t* steps, int64_t* max_per_step,
                                 int64_t* not_converged);

/*
 * Learned initial guess for the GMRES solve (an extension: the paper solves with T_0 directly).
 * For unknown m of right-hand side r at step n the features are x = (y_{n-1}, ..., y_{n-8})_{r,m} / s,
 * s = RMS over edges of y_{n-1} for that r (1 if zero), and the guess is base + s f(x), base = y_{n-1}
 * (TDCFIE_GUESS_MLP) or the cubic extrapolation 4 y_{n-1} - 6 y_{n-2} + 4 y_{n-3} - y_{n-4}
 * (TDCFIE_GUESS_MLP_EXTRAP): the network predicts the correction to its base, so a zero network
 * gives the base itself, with
 *   f(x) = w3 . tanh(W2 tanh(W1 x + b1) + b2) + b3,  W1 64 x 8, W2 64 x 64, w3 64.
 * Parameters: 4801 float32 in the order W1 (row-major), b1, W2 (row-major), b2, w3, b3.
 * Samples: X n x 8 float32 features (row-major), Y n float32 targets.
 */
#define TDCFIE_MLP_NPARAM 4801

/* Gradient of the loss (1/2n) sum_s (f(X_s) - Y_s)^2 at params (all DEVICE pointers): grad receives
 * 4801 floats, loss one float.  FP32 arithmetic.  Enqueued on stream (NULL = legacy stream). */
tdcfie_status tdcfie_mlp_grad(const float* params, const float* X, const float* Y, int64_t n, float* grad,
                              float* loss, void* stream);

/* Adam (beta 0.9 / 0.999, eps 1e-8, rate lr) on the same loss over mini-batches of `batch` samples
 * for `epochs` passes; each pass starts at a seeded rotation of the sample order.  params (DEVICE)
 * is updated in place; loss_history (HOST, epochs floats, or NULL) receives each pass's mean
 * mini-batch loss and makes the call synchronous.  Allocates its optimiser state from the stream's
 * pool and frees it before returning. */
tdcfie_status tdcfie_mlp_train(float* params, const float* X, const float* Y, int64_t n, int epochs, int64_t batch,
                               float lr, uint64_t seed, float* loss_history, void* stream);

/* out[s] = f(X_s) with the weights rounded to float16 (the form used inside the march), FP32
 * arithmetic; DEVICE pointers. */
tdcfie_status tdcfie_mlp_predict(const float* params, const float* X, int64_t n, float* out, void* stream);

/* Training samples from a stored march: y (DEVICE, nt x R x N_E, float64 for precision
 * TDCFIE_FP64 or float32 for TDCFIE_FP32, as written by tdcfie_step_y).  For t = 8 .. nt-1 (0-based
 * rows of y) and every r, m, sample s = ((t - 8) R + r) N_E + m gets X[s] = (y[t-1] .. y[t-8])_{r,m} / sc
 * and Y[s] = (y[t] - base_t)_{r,m} / sc, sc = RMS over edges of y[t-1]_r (1 if zero), base_t = y[t-1]
 * (base 0) or 4 y[t-1] - 6 y[t-2] + 4 y[t-3] - y[t-4] (base 1); the difference is formed in the
 * precision of y: the features the march evaluates before each GMRES solve.  X (DEVICE) holds
 * (nt - 8) R N_E x 8 floats, Y (nt - 8) R N_E.  Needs nt >= 9. */
tdcfie_status tdcfie_mlp_samples(int precision, int base, const void* y, int64_t nt, int64_t R, int64_t ne, float* X,
                                 float* Y, void* stream);

/* Load network parameters (HOST, 4801 floats) into an assembled handle (K - 1 >= 8); they are used
 * while the solver is GMRES with guess TDCFIE_GUESS_MLP.  Synchronous.  Until loaded the weights are
 * zero, so the guess is the previous step. */
tdcfie_status tdcfie_mlp_load(tdcfie_t h, const float* params);

/* Rebuild the step plan of an assembled handle for another path precision and number of
 * right-hand sides (same limits as tdcfie_create) without assembling again: the FP64 blocks are
 * converted anew.  FP64 needs a handle assembled with precision FP64 (the reduced paths form the
 * T_k products in FP32).  The excitation must be set again; a tensor-core plan uses the direct
 * solve. */
tdcfie_status tdcfie_replan(tdcfie_t h, int precision, int64_t max_rhs);

/* Change the per-step solve of an assembled handle (FP64 and FP32 paths for GMRES): solver, initial
 * guess and GMRES tolerance as in tdcfie_opts.  The march state is kept; the step graph is captured
 * again at the next step.  GMRES statistics keep accumulating until the next set_excitation. */
tdcfie_status tdcfie_set_solver(tdcfie_t h, int solver, int guess, double gmres_tol);

/* How the history sum of the FP64 and FP32 paths is streamed (Sec. IV-A, Eq. dis_TD_CFIE):
 *   TDCFIE_HISTORY_DENSE     the dense blocks T_k, k = 1..K-1, multiplied out at assembly (default);
 *   TDCFIE_HISTORY_FACTORED  the shell-sparse retarded matrices S_k, MM_k (+ G/2 at k = 0) and Phi_k
 *     (all lags of a row in one compressed row, lag and column packed in 32 bits), applied to rings of
 *     the physical currents j_i (Eq. post_processing) and the charges Sigma^T y_i, followed per step by
 *     one dense product with W = T_0^-1 [-A | alpha L2 | -L1 Sigma] (formed once in FP64) and by the
 *     projector pair with the dual-graph Laplacian pseudo-inverse.  Same recurrence, other association:
 *     it streams about sum_k nnz(shells) + 3.1 N^2 entries per step instead of (K + 2) N^2.
 * tdcfie_set_history_form rebuilds the step plan of an assembled handle (the excitation must be set
 * again); tdcfie_replan keeps the form (the tensor-core paths always stream dense blocks).  FACTORED needs the FP64 or FP32 path, the direct solve, K <= 256, fewer than 2^24 edges and
 * the FP64 assembly (not released); the FP64 path also needs a handle assembled with precision FP64.
 * TDCFIE_E_UNSUPPORTED / TDCFIE_E_STATE otherwise, and the handle keeps no plan after a failed rebuild.
 * tdcfie_history_stats (host outputs, any may be NULL): the form of the current plan, the nonzeros of
 * the shells (0 for the dense form), the algorithmic bytes per step of the history kernels and of all
 * matrices the step streams. */
typedef enum { TDCFIE_HISTORY_DENSE = 0, TDCFIE_HISTORY_FACTORED = 1 } tdcfie_history_form;
tdcfie_status tdcfie_set_history_form(tdcfie_t h, int form);
tdcfie_status tdcfie_history_stats(tdcfie_t h, int32_t* form, int64_t* nnz, double* history_bytes,
                                   double* step_bytes);

/*
 * Several scatterers marched together (the uneven-batch case; the paper marches one scatterer).
 * Every tdcfie_batch_step advances all handles by one launch of a CUDA graph captured at the first
 * step, and each handle computes exactly what tdcfie_step computes on it (bit for bit).
 *   Persistent form, used when every handle is FP32 with one incident wave and the direct solve:
 *   the graph holds ONE cooperative kernel that walks a work list of all handles' items
 *   (plane-wave tests, per-block history partial sums of 8 rows x 4 blocks, their reduction in
 *   block order, T_0^-1 rows, projector gathers, pseudo-inverse rows, post-processing), longest
 *   items first, with a bounded grid-wide barrier between the seven phases.
 *   Graph-branch form, for any other mix: one step of every handle on its own stream branch.
 *
 * tdcfie_batch_create: handles (host array of n assembled handles on one device, each at most once)
 * are borrowed, not owned: destroy the batch before any of them, and re-create it after
 * tdcfie_replan or tdcfie_set_solver on a member.  Host work plus the work lists' upload.
 * tdcfie_batch_step: every handle must have its excitation set; currents_out is NULL (discard) or a
 * host array of n DEVICE pointers laid out as in tdcfie_step for each handle (entries may be NULL).
 * Synchronous; a member's non-finite current or device timeout is returned with its index.
 * tdcfie_batch_tune (persistent form): times every candidate launch shape (rows per warp 1/2/4,
 * 128/256/512 threads per block, 1/2/4 blocks per SM within the occupancy limit) for
 * steps_per_candidate steps each and keeps the fastest; the candidates march the members, which
 * are then reset to the start of their march (as tdcfie_set_excitation does).  config (host, 4
 * int32, may be NULL) receives {persistent 1/0, rows per warp, threads per block, blocks per SM}.
 * For the graph-branch form it only reports {0, ...}.
 * tdcfie_batch_timing: device time per batch step of the last call and kernel launches per step.
 */
typedef struct tdcfie_batch_s* tdcfie_batch_t;
tdcfie_status tdcfie_batch_create(const tdcfie_t* handles, int64_t n, tdcfie_batch_t* out);
tdcfie_status tdcfie_batch_step(tdcfie_batch_t b, int64_t nsteps, void* const* currents_out);
tdcfie_status tdcfie_batch_tune(tdcfie_batch_t b, int64_t steps_per_candidate, int32_t* config);
tdcfie_status tdcfie_batch_timing(tdcfie_batch_t b, double* step_ms, int64_t* launches_per_step);
tdcfie_status tdcfie_batch_destroy(tdcfie_batch_t b);

/* The system the step marches.  TDCFIE_FORMULATION_QHP_CFIE (default): the qHP TD-CFIE of
 * Eq. qHP_TDCFIE.  TDCFIE_FORMULATION_MFIE: the mixed TD-MFIE, one of the paper's comparison
 * formulations (Sec. V), (G/2 + MM) j = h with the hat basis in time and Dirac testing on the same
 * matrices: sum_k MM'_k j_{n-k} = h_n, MM'_k = MM_k + G/2 [k = 0]; the currents are j directly.
 * tdcfie_set_formulation rebuilds the plan of an assembled handle (excitation to be set again);
 * MFIE needs the dense FP64 or FP32 path with the direct solve and the FP64 assembly (not
 * released): TDCFIE_E_UNSUPPORTED / TDCFIE_E_STATE otherwise; the formulation is kept by
 * tdcfie_replan, which then refuses the tensor-core paths, as set_history_form and set_solver
 * refuse the factored form and GMRES. */
typedef enum { TDCFIE_FORMULATION_QHP_CFIE = 0, TDCFIE_FORMULATION_MFIE = 1 } tdcfie_formulation;
tdcfie_status tdcfie_set_formulation(tdcfie_t h, int formulation);

/* Far field of marched currents at angular frequency w (Sec. V, the large-time-step test compares
 * the sphere's far field at 3 Hz with the series solution); units c = eta = mu = 1, phasors e^{j w t}:
 *   J_m(w) = dt sinc^2(w dt / 2) sum_i j_m[i] e^{-j w t_i}   (hat basis of Eq. post_processing, t_i = i dt)
 *   F(rhat) = -j w / (4 pi) (I - rhat rhat) sum_m J_m(w) int f_m(r) e^{j w rhat.r} dS   (7-point rule)
 * so that the scattered field is F e^{-j w r} / r.  currents: DEVICE, nt x R x ne as written by
 * tdcfie_step from the march's first step (path precision: FP64 on the FP64 path, FP32 otherwise);
 * rhat: HOST ndir x 3 unit vectors (ndir <= 65535); out: HOST ndir x R x 3 x 2 doubles (re, im).
 * FP64 arithmetic; synchronous on the handle's stream; TDCFIE_E_ARG for bad arguments. */
tdcfie_status tdcfie_far_field(tdcfie_t h, const void* currents, int64_t nt, double w, const double* rhat,
                               int64_t ndir, double* out);

/* Whole march: set_excitation, then nt steps into currents_out.  out_on_host != 0: currents_out is a
 * HOST buffer (pinned or pageable) and the device-to-host copy is part of the call. */
tdcfie_status tdcfie_march(tdcfie_t h, const tdcfie_plane_waves* exc, void* currents_out, int out_on_host);

/* Sizes of the discretisation. Any pointer may be NULL. */
tdcfie_status tdcfie_info(tdcfie_t h, int64_t* ne, int64_t* nc, int64_t* nv, int64_t* K, int32_t* genus,
                          double* D);

/* Edge table for bit-exact checks: edges ne x 2 (v-, v+), cplus / cminus ne (host outputs). */
tdcfie_status tdcfie_topology(tdcfie_t h, int32_t* edges, int32_t* cplus, int32_t* cminus);

/* BC coefficient table of the barycentric refinement (Sec. II-C, Fig. 2), host outputs:
 * nentries; per entry the fine triangle, the BC function (edge) and the three outward fluxes
 * through the fine triangle's edges opposite its vertices 0, 1, 2 (g_n = sum_j phi_j (r - w_j)/(2A));
 * fine_vertices (nv + ne + nc) x 3 (vertices, edge midpoints, barycentres); fine_triangles
 * (6 nc) x 3.  Any output may be NULL (query nentries first). */
tdcfie_status tdcfie_bc_table(tdcfie_t h, int64_t* nentries, int32_t* fine_tri, int32_t* fn, double* phi,
                              double* fine_vertices, int32_t* fine_triangles);

/* Copy an assembled FP64 matrix to a host buffer (row-major):
 *   which 0: T_k (ne x ne), 1: S_k (ne x ne), 2: H_k (ne x ne), 3: MM_k (ne x ne),
 *   4: G, 5: Z^s, 6: Z^h, 7: M, 8: P^Sigma, 9: L1, 10: L2 (ne x ne; k ignored),
 *   11: Phi_k (nc x nc, the charge-potential matrix with H_k = Sigma Phi_k Sigma^T). */
tdcfie_status tdcfie_get_matrix(tdcfie_t h, int which, int64_t k, double* host_out);

/* Device time (ms, CUDA events on the handle's stream) of the last tdcfie_step call and of its
 * history-sum kernels alone; history_bytes = algorithmic bytes those kernels stream per step. */
tdcfie_status tdcfie_last_timing(tdcfie_t h, double* step_ms, double* history_ms, double* history_bytes,
                                 int64_t* kernel_launches);

/*
 * Stand-alone history sum of the MOT recurrence (Sec. IV-B, the sum over k of T_k y_{n-k}) for
 * blocks the caller holds:
 *     out[r][i] = sum_{q < nblk} sum_{j < n} blocks[q][i][j] x[q][r][j]
 * blocks: DEVICE, nblk x n x n, row-major; x: DEVICE, nblk x R x n (block q's R vectors);
 * out: DEVICE, R x n.  Element type double for TDCFIE_FP64 and float for TDCFIE_FP32 (FP32
 * accumulation); 1 <= nblk <= 65535, 1 <= n <= 2^24, 1 <= R <= 8.  Per-block partial sums go to
 * scratch taken with cudaMallocAsync / cudaFreeAsync on `stream` (cudaStream_t, NULL = legacy
 * default stream); the blocks are then added in a fixed order, so results are deterministic.
 * Asynchronous: returns after queueing.  Errors: TDCFIE_E_ARG, TDCFIE_E_UNSUPPORTED,
 * TDCFIE_E_OOM, TDCFIE_E_CUDA (thread-local message in tdcfie_last_error(NULL)).
 */
tdcfie_status tdcfie_block_gemv(int precision, const void* blocks, int64_t nblk, int64_t n, const void* x, int64_t R,
                                void* out, void* stream);

/*
 * tdcfie_block_gemv for callers that cannot allocate device memory at the time of the call (for
 * example a thread of a process in which another thread holds a global-mode stream capture, a
 * service whose allocator has reserved nearly all device memory, or a loop that cannot take an
 * allocation's implicit synchronisation).  The paper has no counterpart; this is a library
 * service.  Same arguments, layouts, arithmetic and result as tdcfie_block_gemv, but the
 * per-block partial sums go to a file-scope static device array of 32 MiB that every GPU loading
 * the library holds until the process exits: nblk * R * n must not exceed 4194304 (FP64) or
 * 8388608 (FP32), else TDCFIE_E_ARG with a message.  No cudaMalloc, cudaFree or allocating
 * library routine is called.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call before any stream
 * capture.  All calls share the one array and every partial sum a call reads it has written
 * first, so nothing needs clearing between calls; calls whose executions overlap on the GPU
 * (different streams, or graphs replayed concurrently) race on it and must be serialised.
 */
tdcfie_status tdcfie_block_gemv_noalloc(int precision, const void* blocks, int64_t nblk, int64_t n, const void* x,
                                        int64_t R, void* out, void* stream);

/*
 * The history sum of the MOT recurrence (Sec. IV-B, the sum over k of T_k y_{n-k}) in the split
 * tensor-core arithmetic of the FP16X3 / BF16X3 paths, for caller-held blocks:
 *     out[r][i] = sum_{q < nblk} sum_{j < cols} blocks[q][i][j] x[q][r][j]
 * blocks: DEVICE, nblk x rows x cols float64, row-major; x: DEVICE, nblk x R x cols float64;
 * out: DEVICE, R x rows float64 (caller-owned).  R must be 64.  The blocks are split into two
 * 16-bit slices with one power-of-two scale per row, the vectors into three (FP16X3) or two
 * (BF16X3) slices with one scale per 64-element tile, exactly as inside tdcfie_step; the partial
 * sums are added in FP64.  1 <= nblk <= 4096, 1 <= rows, cols <= 2^20.  Takes its scratch with
 * cudaMalloc and frees it before returning; synchronous on `stream` (cudaStream_t, NULL = legacy
 * default stream).  Errors: TDCFIE_E_ARG, TDCFIE_E_UNSUPPORTED, TDCFIE_E_OOM, TDCFIE_E_CUDA,
 * TDCFIE_E_TIMEOUT (thread-local message in tdcfie_last_error(NULL)).
 */
tdcfie_status tdcfie_tc_gemm(int precision, const double* blocks, int64_t nblk, int64_t rows, int64_t cols,
                             const double* x, int64_t R, double* out, void* stream);

/* Wall-clock seconds of the phases of the last tdcfie_assemble (host output, 6 values): mesh upload,
 * retarded EFIE quadrature, retarded MFIE quadrature, static quadrature, formation of the blocks
 * (projectors, preconditioner, T_k, inverses), path-precision copies. */
tdcfie_status tdcfie_assembly_timing(tdcfie_t h, double* seconds);

/* Free the FP64 assembly matrices of an assembled handle (S_k, Phi_k, MM_k, H_k, T_k, the static
 * matrices, L1, L2, the FP64 T_0^-1) and keep only the current step plan, for batches of large
 * scatterers whose FP64 assembly would not fit on the device together.  The march is unaffected;
 * afterwards tdcfie_replan, tdcfie_get_matrix and switching to GMRES (unless its T_0 copy already
 * exists) return TDCFIE_E_STATE.  Synchronous.  Errors: TDCFIE_E_ARG, TDCFIE_E_STATE, TDCFIE_E_CUDA. */
tdcfie_status tdcfie_release_assembly(tdcfie_t h);

tdcfie_status tdcfie_destroy(tdcfie_t h);

/* Message of the last error of h (thread-local last error when h is NULL). Never NULL. */
const char* tdcfie_last_error(tdcfie_t h);

#ifdef __cplusplus
}
#endif
#endif /* TDCFIE_H */
