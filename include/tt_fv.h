/*
 * tt_fv.h -- C ABI of the GB300 tensor-train finite-volume shallow-water stage.
 *
 * Method: Danis, Truong, DeSantis, Petersen, Rasmussen, Alexandrov,
 * "High-order Tensor-Train Finite Volume Method for Shallow Water Equations",
 * arXiv 2408.03483.  Section / equation / algorithm numbers below refer to it.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - A 2-D TT ("matrix TT", Sec. 3.1, Eq. TT_def_2D) is a pair of cores:
 *       X[i, j] = sum_{k < rank} a[k * n1 + i] * b[k * n2 + j],
 *   i.e. a = G1 (n1 x rank, column-major, i fastest) and b = G2^T
 *   (n2 x rank, column-major).  The first index is x, the second y.
 * - Every pointer in a tt2 is DEVICE memory owned by the caller, sized for
 *   `cap` columns (a: n1 * cap doubles, b: n2 * cap doubles).  The library
 *   never allocates, frees or keeps caller memory beyond a call, except the
 *   workspace handed to tt_fv_init, which the context uses until destroy.
 * - `ws` / `ws_bytes`: caller-provided device workspace (>= the size the
 *   matching *_workspace_size function returns; 256-byte aligned).
 * - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *   stream-ordered; a call returns after its last launch and may read a few
 *   integers back from the device (ranks, iteration counts) on that stream.
 * - Errors are return codes only; nothing aborts or traps.  TT_ERR_ARG: bad
 *   argument (no work done); TT_ERR_OOM: workspace too small; TT_ERR_CUDA: a
 *   CUDA call failed; TT_ERR_NOCONV: an iteration hit its cap (Taylor
 *   reciprocal, Jacobi SVD); the output is then the last iterate.
 *   TT_ERR_NONFINITE: a NaN or Inf reached a small SVD or maxvol (the
 *   kernels then produce a harmless placeholder instead of indexing with
 *   it); TT_ERR_TIMEOUT: a tensor-core kernel's bounded wait expired.
 *   Reaching a rank cap truncates to the cap and is counted, not an error.
 * - Arithmetic: IEEE FP64 throughout in the plain path (precision TT_FP64);
 *   the precision forms (TT_FP32, TT_TF32, TT_BF16) run the rounding
 *   contractions in FP32 on CUDA cores or on tcgen05 tensor cores with FP32
 *   accumulation (split operands, FP32-accurate), while the small SVDs,
 *   maxvol's choices of rows, the Taylor scaling and every stored core stay
 *   FP64; tt_contract exposes the contraction in each precision.
 */
#ifndef TT_FV_H
#define TT_FV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TT_OK = 0,
  TT_ERR_ARG = 1,
  TT_ERR_OOM = 2,
  TT_ERR_CUDA = 3,
  TT_ERR_NOCONV = 4,
  TT_ERR_TIMEOUT = 5,
  TT_ERR_RANKCAP = 6,
  TT_ERR_NONFINITE = 7
} tt_status;

typedef struct {
  int32_t n1, n2;   /* mode sizes */
  int32_t rank;     /* current rank (columns in use) */
  int32_t cap;      /* allocated columns */
  double* a;        /* n1 x cap, device */
  double* b;        /* n2 x cap, device */
} tt2;

enum { TT_LINEAR = 0, TT_NONLINEAR = 1 };          /* Eq. linear-SWE / nonlinear-SWE */
enum { TT_UP3 = 0, TT_UP5 = 1, TT_WENO5 = 2 };      /* Sec. 2.3 reconstructions */
enum { TT_FP64 = 0, TT_TF32 = 1, TT_BF16 = 2, TT_FP32 = 3 }; /* contraction precision */
enum { TT_PIVOT_MAXVOL = 0, TT_PIVOT_LEARNED = 1 };
enum { TT_EPS_FIXED = 0, TT_EPS_ADAPTIVE = 1 };       /* truncation tolerance rule (Sec. 4.4) */

/* Cross-interpolated functions (tt_cross `fn`). */
enum {
  TT_FN_ENTRY = 0,       /* F = inputs[0] itself (exact-recovery test)              */
  TT_FN_WENO_S1 = 1,     /* WENO5 Step 1 (Sec. 2.3.1, Algorithm 2) of inputs[0]     */
  TT_FN_WENO_S2 = 2,     /* WENO5 Step 2 at all Gauss points (Algorithm 3)          */
  TT_FN_LLF_LAMBDA = 3,  /* max(|hu-/h-| + sqrt(g h-), |hu+/h+| + sqrt(g h+)) (Sec. 4.2) */
  TT_FN_LLF_FLUX = 4     /* the LLF flux vector of Eq. LLF from the face states, its three
                            components stacked along the first mode (the LF-cross of Sec. 4.2) */
};
enum { TT_FLUX_PRODUCTS = 0, TT_FLUX_CROSS = 1 }; /* nonlinear LLF flux in TT (Sec. 4.2) */
enum { TT_BC_PERIODIC = 0, TT_BC_EXACT = 1 };     /* x boundary (Sec. 5.1, 5.3) */

typedef struct {
  int32_t eqn;        /* TT_LINEAR | TT_NONLINEAR */
  int32_t recon;      /* TT_UP3 | TT_UP5 | TT_WENO5 */
  int32_t nx, ny;     /* cells; domain [0,lx] x [0,ly], doubly periodic */
  double lx, ly;
  double g, H, f;     /* gravity, mean depth (linear SWE), Coriolis parameter */
  double dt;          /* time step */
  double tol;         /* relative Frobenius truncation tolerance of every round */
  int32_t rank_cap;   /* rank cap of every round */
  int32_t precision;  /* TT_FP64 (plain), or a precision form: TT_FP32 (FP32 rounding contractions on CUDA
                         cores), TT_TF32 / TT_BF16 (their large products on tcgen05 with split operands);
                         SVDs and stored cores stay FP64 */
  int32_t pivots;     /* TT_PIVOT_MAXVOL, or TT_PIVOT_LEARNED: crosses start from the pivots of the
                         network set by tt_fv_set_pivot_net (maxvol start until one is set) */
  int32_t kick;       /* cross kick fibres per sweep (default 4 if <= 0) */
  int32_t max_sweeps; /* cross sweep cap (default 10 if <= 0) */
  int32_t max_iter;   /* Taylor reciprocal iteration cap (default 50 if <= 0) */
  uint32_t seed;      /* seed of the cross kick indices */
  int32_t eps_rule;   /* TT_EPS_FIXED (0): `tol` for every round and cross.  TT_EPS_ADAPTIVE (Sec. 4.4):
                         at the start of each step, from the step's input state,
                           eps_u  = min(1e-3, c_eps V^(1/2) dx^(p-1/2) / ||u||_F)   per field u, for its
                                    forward-Euler and SSP-combination rounds (Eq. modified-eps-tt-formula),
                           eps_TT = c_eps V^(1/2) dx^(p-1/2) / max_q ||q||_F        for every other round
                                    and cross (Eq. eps-tt-formula),
                         with V = lx ly, dx = lx / nx, p = 3 (TT_UP3) or 5; `tol` is then unused */
  double c_eps;       /* C_eps of Sec. 4.4 (> 0 under TT_EPS_ADAPTIVE; Table 1 gives the paper's values) */
  int32_t flux;       /* nonlinear SWE, how Eq. LLF-TT is formed (Sec. 4.2): TT_FLUX_PRODUCTS (0): 1/h by
                         Algorithm 1, the physical fluxes from rounded Hadamard products, lambda by cross,
                         then the rounded LLF sums; TT_FLUX_CROSS: per direction one cross of the whole
                         flux vector (TT_FN_LLF_FLUX), the LF-cross the paper compares against */
  int32_t forcing_waves; /* the most source waves of one field tt_fv_set_forcing may set, 0..TT_MAX_WAVES
                            (0: no source); the workspace is sized for it */
  int32_t bc_x;       /* TT_BC_PERIODIC (0), or TT_BC_EXACT: the domain is bounded in x and the three
                         cells beyond each x boundary hold the exact solution set by tt_fv_set_boundary
                         (the linear SWE with TT_UP3 / TT_UP5 only); y stays periodic */
  int32_t boundary_waves; /* under TT_BC_EXACT: the most plane waves of one field of that exact
                             solution, 1..TT_MAX_WAVES; the workspace is sized for it */
} tt_fv_params;

/* One wave amp exp(-decay x) cos(kx x + ky y - omega t + phase) of field
 * `field` (0: h or eta, 1: hu or u, 2: hv or v): a plane wave when decay = 0,
 * e.g. a term of the forcing that makes the manufactured solution of Sec. 5.4
 * exact or of the barotropic tide of Sec. 5.3; damped in x when decay > 0,
 * e.g. a term of the coastal Kelvin wave of Sec. 5.1 (decay = 1/R).  Its cell
 * averages are exact: the y factor's centre value times sinc(ky dy/2), the x
 * factors' from the integral of exp((-decay + i kx) x) over the cell. */
typedef struct {
  int32_t field;
  double amp, kx, ky, omega, phase;
  double decay;
} tt_wave;
enum { TT_MAX_WAVES = 16 };

typedef struct {
  int32_t rank[3];            /* current ranks of the three fields */
  int64_t rounds;             /* TT roundings performed */
  int64_t syncs;              /* device->host reads of ranks / counters */
  int64_t jacobi_sweeps;      /* sweeps of the small SVDs */
  int64_t cross_calls, cross_sweeps;
  int64_t taylor_iters;       /* Algorithm 1 loop iterations */
  int64_t cap_hits;           /* rounds truncated by the rank cap */
  int64_t qb_attempts, qb_uncertified;  /* range-finder attempts / residual above target */
  double flops;               /* algorithmic FP64 flops issued */
  double bytes;               /* algorithmic bytes moved by the core kernels */
  uint32_t device_status;     /* latched device error bits (0 = none) */
  int64_t svd_calls;          /* small SVDs */
  int64_t svd_p_sum;          /* sum of their sizes p */
  int64_t svd_pd_sum;         /* sum of their deflated ranks */
  int64_t svd_sweeps_sum;     /* sum of their Jacobi sweeps */
  double section_ms[6];       /* host wall time per stage section: faces, side fluxes + lambda,
                                 LLF combination, quadrature/difference, forward-Euler rounds,
                                 SSP combination rounds.  The nonlinear stage runs as one
                                 dependency graph whose phases overlap: there the first five
                                 are how far each phase's last task finished after the
                                 previous phase's (they add up to the graph's wall time) */
  int64_t learned_calls;      /* crosses started from the learned network's pivots */
  int64_t learned_accepted;   /* ... whose first interpolation check passed (no maxvol fallback) */
  double eps_u[3];            /* tolerances of the current step's per-field rounds (Sec. 4.4) */
  double eps_tt;              /* tolerance of the current step's other rounds and crosses */
} tt_fv_stats;

typedef struct tt_fv_ctx tt_fv_ctx;

/* Kernel classes of the per-launch profile (tt_fv_kernel_profile). */
enum {
  TT_K_GEMM = 0,      /* FP64 split-K GEMM (range finder, factor products)     */
  TT_K_FORM = 1,      /* full Hadamard face tensor formation                   */
  TT_K_QR = 2,        /* Householder TSQR row blocks (leaves)                  */
  TT_K_QR_APPLY = 3,  /* application of the leaves' orthogonal factors         */
  TT_K_JACOBI = 4,    /* one-sided Jacobi SVD of the small core                */
  TT_K_MAXVOL = 5,    /* maximum-volume row selection                          */
  TT_K_EVAL = 6,      /* cross fibre evaluation (WENO5, LLF speed)             */
  TT_K_STENCIL = 7,   /* core stencils: reconstruction, quadrature, (T-1)/dx   */
  TT_K_OTHER = 8,     /* copies, transposes, norms, small solves               */
  TT_K_QR_MERGE = 9,  /* TSQR merges of stacked triangular factors              */
  TT_K_QR_APPLY_MERGE = 10, /* application of the merges' orthogonal factors    */
  TT_K_NCLASS = 11
};

typedef struct {
  double ms;          /* summed device time of the launches (CUDA events)      */
  double flops;       /* algorithmic FP64 flops of those launches              */
  double bytes;       /* algorithmic DRAM bytes of those launches              */
  int64_t launches;
} tt_kernel_prof;

/* ---------------------------------------------------------------- solver */

/* Device workspace needed by tt_fv_init for these parameters (bytes). */
size_t tt_fv_workspace_size(const tt_fv_params* p);

/* Create a solver context: copies the initial fields q0 (h, hu, hv for the
 * nonlinear SWE; eta, u, v for the linear SWE; cell averages in TT format,
 * ranks <= rank_cap, n1 = nx, n2 = ny) into state held in `ws`.  The context
 * keeps using `ws` (caller-owned) until tt_fv_destroy. */
tt_status tt_fv_init(const tt_fv_params* p, const tt2 q0[3], void* ws, size_t ws_bytes,
                     void* stream, tt_fv_ctx** out);

/* nsteps full SSP-RK3 steps (Eq. tt-ssprk3 with Eq. tt-forward-euler). */
tt_status tt_fv_step(tt_fv_ctx* ctx, int32_t nsteps);

/* One SSP-RK3 stage: stage 0 sets u1 = F(u^n); stage 1 sets
 * u2 = round(3/4 u^n + 1/4 F(u1)); stage 2 sets u^{n+1} = round(1/3 u^n + 2/3 F(u2))
 * and makes it the new u^n.  Stages must be called in order 0, 1, 2. */
tt_status tt_fv_stage(tt_fv_ctx* ctx, int32_t stage);

/* Copy the current state (u^n after a full step, or the latest stage value)
 * into caller cores (cap >= rank, n1/n2 matching); sets q_out[c].rank. */
tt_status tt_fv_get(tt_fv_ctx* ctx, tt2 q_out[3]);

/* Replace u^n by caller cores (checkpoint resume). */
tt_status tt_fv_set(tt_fv_ctx* ctx, const tt2 q[3]);

/* Sets the external source of a solver (method of manufactured solutions,
 * Sec. 5.4): `nwaves` plane waves (host array, copied; at most
 * params.forcing_waves per field, else TT_ERR_ARG).  Each stage evaluates
 * them as exact cell averages -- the centre value times sinc(kx dx/2)
 * sinc(ky dy/2), a rank-2 TT per wave -- at its own time (t, t + dt,
 * t + dt/2 for the three stages of Eq. tt-ssprk3) and adds dt times them to
 * u + dt L(u) before the forward-Euler round.  t0 is the time of the current
 * state; each step advances it by dt.  nwaves = 0 removes the source. */
tt_status tt_fv_set_forcing(tt_fv_ctx* ctx, const tt_wave* waves, int32_t nwaves, double t0);

/* Sets the exact solution that supplies the x-boundary values of a solver with
 * bc_x = TT_BC_EXACT (the exact-solution boundary of Sec. 5.1 and Sec. 5.3):
 * `nwaves` plane waves (host array, copied; at most params.boundary_waves per
 * field, else TT_ERR_ARG).  At each stage's time (t, t + dt, t + dt/2) the
 * three cells beyond x = 0 and beyond x = lx take the waves' exact cell
 * averages: every field's TT is extended by those ghost rows (its first core
 * by rank-2-per-wave columns that are zero on the real rows, its second core
 * by the waves' y factors), Step 1 and Step 2 in x run without wrapping, the
 * x faces are the nx + 1 faces x_{-1/2} .. x_{nx-1/2}, and the flux difference
 * in x does not wrap.  t0 is the time of the current state (shared with the
 * source of tt_fv_set_forcing).  A solver with TT_BC_EXACT refuses to step
 * (TT_ERR_ARG) until its boundary is set. */
tt_status tt_fv_set_boundary(tt_fv_ctx* ctx, const tt_wave* waves, int32_t nwaves, double t0);

tt_status tt_fv_stats_get(tt_fv_ctx* ctx, tt_fv_stats* out);
void tt_fv_destroy(tt_fv_ctx* ctx);

/* TSQR tile shapes of the rounding (Sec. 3.2's QR of the cores, done as a
 * tree of leaf QRs and merges): shape s is (leaf_mult[s], fanin[s]), the leaf
 * rows as a multiple of max(64, rank rounded up to 32) and the largest merge
 * fan-in (0: the default 4), both capped by shared memory.  tt_tile_shapes
 * writes up to `max` shapes (either array may be NULL) and returns their
 * number; shape 0, (2, 0), is the default of every entry point.  tt_fv_workspace_size covers every shape.
 * tt_fv_set_tile_shape switches a solver's roundings to shape `shape`
 * (results change at round-off level only); TT_ERR_ARG for an unknown shape. */
int32_t tt_tile_shapes(int32_t* leaf_mult, int32_t* fanin, int32_t max);
tt_status tt_fv_set_tile_shape(tt_fv_ctx* ctx, int32_t shape);

/* Enable (1) or disable (0) CUDA-event timing of every kernel launch of the
 * context, accumulated per kernel class.  While enabled, the stage's
 * independent tasks run one after another on the context stream (so a
 * launch's time is its own device time) and two events are recorded per
 * launch: a profiled stage is slower than an unprofiled one. */
tt_status tt_fv_profile(tt_fv_ctx* ctx, int32_t enable);
/* Copy the accumulated per-class profile (TT_K_NCLASS entries) and, if
 * reset != 0, clear it. */
tt_status tt_fv_kernel_profile(tt_fv_ctx* ctx, tt_kernel_prof out[TT_K_NCLASS], int32_t reset);
/* Kernels launched by this library in this process so far. */
uint64_t tt_launch_count(void);

/* ---------------------------------------------------------------- primitives */

/* TT rounding (Sec. 3.2): y = round(x, tol) with rank <= rank_cap, the
 * truncated SVD of X at relative Frobenius tolerance tol (keep the smallest k
 * with sqrt(sum_{i>k} s_i^2) <= tol ||X||_F, then min(k, rank_cap), k >= 1).
 * y->a / y->b must not alias x; y->cap >= rank_cap.  err_out (host, may be
 * NULL) receives the discarded Frobenius norm. */
size_t tt_round_workspace_size(int32_t n1, int32_t n2, int32_t rank_in, int32_t rank_cap);
tt_status tt_round(const tt2* x, double tol, int32_t rank_cap, tt2* y, double* err_out,
                   void* ws, size_t ws_bytes, void* stream);

/* Learned-pivot form.  The paper's crosses (Sec. 3.3) refine pivots by maxvol
 * sweeps from some start; this form starts them from the column indices that
 * a 3-layer perceptron (14 -> 256 -> 256 -> 1, ReLU) scores highest from
 * features of the cross's initial TT and of the call site's previous pivots,
 * and accepts them after one sweep when that sweep's skeleton already
 * predicts fresh sample rows to the tolerance.  The sweeps still judge the sampled
 * interpolation error against the tolerance, so plain maxvol refinement is
 * the fallback whenever the proposal is not good enough.
 *   tt_mlp: caller-owned device FP32 parameters: W1 14x256 and W2 256x256
 *   row-major (W[in*256 + out]), b1, b2, w3 (256 each), b3 (1).  Every
 *   product of the forward and backward passes runs on tcgen05 tensor cores
 *   with both operands rounded to BF16 and FP32 accumulation.
 *   tt_mlp_features: X (n2 x 14 column-major, ld n2, device float) = the index
 *   features of x0's column mode (leverage of an orthonormal basis of x0->b
 *   and of its 4 neighbours, standardised column mean and its first/second
 *   differences, log curvature, column energy, sin/cos of the index angle,
 *   and, from the nprev device indices prev of the same cross site's previous
 *   converged pivots, an indicator and the distance to them capped at 8).
 *   tt_mlp_forward: scores s (m) of the rows of X (m x 12, ld m).
 *   tt_mlp_grad: gradients of the mean logistic loss over labels y (m, 0/1)
 *   into *grad (same shapes as net) and the loss into *loss (device double,
 *   may be NULL).  tt_mlp_adam: one Adam step (0.9, 0.999, 1e-8) of net with
 *   moment buffers m1, m2 (zero-initialised by the caller), step t >= 1.
 *   tt_mlp_topk: the k (<= 128) highest scores' indices, ties to the smaller
 *   index, written ascending to idx (device).
 *   Workspace: tt_mlp_workspace_size(rows, rank) covers features of an
 *   n2 = rows TT of that rank and forward/grad/topk over `rows` rows.
 * Solver hooks: tt_fv_set_pivot_net points a TT_PIVOT_LEARNED solver at a
 * network (NULL: back to the maxvol start); tt_fv_record_pivots(ctx, 1)
 * starts capturing, for every cross, the features of its initial TT with
 * label 1 on the converged column pivots (training data; adds a sync per
 * cross), tt_fv_pivot_rows reports the captured rows and tt_fv_pivot_take
 * copies them to host arrays X (rows x 14 row-major) and y (rows), then
 * clears the capture. */
typedef struct {
  float* W1;
  float* b1;
  float* W2;
  float* b2;
  float* w3;
  float* b3;
} tt_mlp;
size_t tt_mlp_workspace_size(int32_t rows, int32_t rank);
tt_status tt_mlp_features(const tt2* x0, const int32_t* prev, int32_t nprev, float* X, void* ws, size_t ws_bytes,
                          void* stream);
tt_status tt_mlp_forward(const tt_mlp* net, const float* X, int32_t m, float* s, void* ws, size_t ws_bytes,
                         void* stream);
tt_status tt_mlp_grad(const tt_mlp* net, const float* X, const float* y, int32_t m, const tt_mlp* grad,
                      double* loss, void* ws, size_t ws_bytes, void* stream);
tt_status tt_mlp_adam(const tt_mlp* net, const tt_mlp* grad, const tt_mlp* m1, const tt_mlp* m2, int32_t t,
                      float lr, void* stream);
tt_status tt_mlp_topk(const float* s, int32_t m, int32_t k, int32_t* idx, void* ws, size_t ws_bytes, void* stream);
tt_status tt_fv_set_pivot_net(tt_fv_ctx* ctx, const tt_mlp* net);
tt_status tt_fv_record_pivots(tt_fv_ctx* ctx, int32_t enable);
int64_t tt_fv_pivot_rows(tt_fv_ctx* ctx);
tt_status tt_fv_pivot_take(tt_fv_ctx* ctx, float* X, float* y, int64_t rows);

/* Batched form: an ensemble of independent solver instances (uneven grid
 * size, rank cap, reconstruction and precision) advanced together on one GPU.
 *   p[count], q0[3*count]: per-instance parameters and initial fields, as for
 *   tt_fv_init (copied at init).  ws: one caller workspace of at least
 *   tt_fv_batch_workspace_size(p, count) bytes, sliced per instance.  Each
 *   instance runs on its own stream, created by the batch; `stream` is the
 *   caller's stream, ordered after all instance work at the end of every
 *   tt_fv_batch_step.
 * tt_fv_batch_step advances every instance by nsteps full SSP-RK3 steps: host
 *   workers take instances longest-first (cost = the instance's previous step
 *   time) so that several instances' kernels share the GPU.
 * tt_fv_batch_configure sets the worker count and whether each instance also
 *   runs its own independent stage tasks concurrently (inner_tasks != 0).
 * tt_fv_batch_tune runs steps_per_trial real batch steps for each candidate
 *   worker count, with inner tasks off and on, keeps the fastest setting and
 *   reports it (the trial steps advance the ensemble); rates (may be NULL,
 *   2*ncand doubles) receives each trial's cell updates per second, index
 *   2*c + inner.
 * tt_fv_batch_tune_tiles times every TSQR tile shape of tt_tile_shapes
 *   (rounds x steps_per_trial real batch steps per shape, the shapes
 *   interleaved round by round, all instances on the same shape in a trial)
 *   and gives each instance the shape of its own least step time; shape_out
 *   (may be NULL, count int32) receives each instance's shape, rates (may be
 *   NULL, one double per shape) the batch's cell updates per second under
 *   each shape.  The trial steps advance the ensemble.
 * tt_fv_batch_get / tt_fv_batch_stats_get: as tt_fv_get / tt_fv_stats_get for
 *   instance i.  Errors: TT_ERR_ARG, TT_ERR_OOM (workspace too small), or the
 *   first error an instance returned. */
typedef struct tt_fv_batch tt_fv_batch;
size_t tt_fv_batch_workspace_size(const tt_fv_params* p, int32_t count);
tt_status tt_fv_batch_init(const tt_fv_params* p, int32_t count, const tt2* q0, void* ws, size_t ws_bytes,
                           void* stream, tt_fv_batch** out);
tt_status tt_fv_batch_configure(tt_fv_batch* b, int32_t workers, int32_t inner_tasks);
tt_status tt_fv_batch_step(tt_fv_batch* b, int32_t nsteps);
tt_status tt_fv_batch_tune(tt_fv_batch* b, const int32_t* workers, int32_t ncand, int32_t steps_per_trial,
                           int32_t* best_workers, int32_t* best_inner, double* rates);
tt_status tt_fv_batch_tune_tiles(tt_fv_batch* b, int32_t steps_per_trial, int32_t rounds, int32_t* shape_out,
                                 double* rates);
tt_status tt_fv_batch_get(tt_fv_batch* b, int32_t i, tt2 q_out[3]);
tt_status tt_fv_batch_stats_get(tt_fv_batch* b, int32_t i, tt_fv_stats* out);
void tt_fv_batch_destroy(tt_fv_batch* b);

/* Dense contraction C = alpha A B + beta C in the working precision of a
 * precision form -- the core-times-factor and face-tensor products of TT
 * rounding (Sec. 3.2) that the precision forms move off FP64.
 *   A: m x k, B: k x n, C: m x n, FP64, column-major device arrays with
 *   leading dimensions lda >= m, ldb >= k, ldc >= m (caller-owned; C is
 *   overwritten, and read when beta != 0).
 *   precision: TT_FP64 (FP64 CUDA cores), TT_FP32 (operands rounded to FP32,
 *   FP32 CUDA-core products), TT_TF32 / TT_BF16 (tcgen05 tensor cores, FP32
 *   accumulation).  split (TF32/BF16 only): nonzero decomposes each operand
 *   into tensor-core parts (TF32: hi + lo, 3 products; BF16: hi + mid + lo,
 *   6 products) whose sum reaches FP32 accuracy; 0 rounds each operand once.
 *   The result is rounded to FP32 before alpha/beta are applied in FP64.
 * Errors: TT_ERR_ARG for bad shapes/pointers/precision; TT_ERR_OOM if ws is
 * smaller than tt_contract_workspace_size(); TT_ERR_TIMEOUT if a tensor-core
 * kernel's bounded wait expired. */
size_t tt_contract_workspace_size(int32_t precision, int32_t split, int32_t m, int32_t n, int32_t k);
tt_status tt_contract(int32_t precision, int32_t split, int32_t m, int32_t n, int32_t k, double alpha,
                      const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                      int64_t ldc, void* ws, size_t ws_bytes, void* stream);

/* tt_round without any device allocation, for callers that cannot allocate
 * device memory (no cudaMalloc available to them, or a fixed memory footprint
 * that must not grow).  The paper has no counterpart: this is a packaging
 * variant of tt_round.  Same arguments and results as tt_round; the scratch is
 * a 32 MiB array in this library's device memory (held by every GPU that loads
 * the library until process exit) instead of a caller workspace, so sizes
 * whose tt_round_workspace_size exceeds 32 MiB are rejected with TT_ERR_ARG.
 * The first call on a device (with that device current) looks up the array's
 * device address; make that first call before any stream capture.  The
 * address is kept for the life of the process: after a cudaDeviceReset the
 * array lives at a new address, so do not call this entry point on a device
 * that was reset in the same process.  Like tt_round, the call waits for its
 * stream before returning (it reads the device status word).  Every call
 * shares the one array and overwrites it: calls that overlap on the GPU (two
 * streams, two threads) race, so serialise them. */
tt_status tt_round_noalloc(const tt2* x, double tol, int32_t rank_cap, tt2* y, double* err_out,
                           void* stream);

/* y = round(x o z, tol): the TT Hadamard product (Sec. 4.2, cores are
 * row-wise Kronecker products of rank x.rank * z.rank) followed by rounding. */
size_t tt_round_hadamard_workspace_size(int32_t n1, int32_t n2, int32_t rank_x, int32_t rank_z,
                                        int32_t rank_cap);
tt_status tt_round_hadamard(const tt2* x, const tt2* z, double tol, int32_t rank_cap, tt2* y,
                            void* ws, size_t ws_bytes, void* stream);

/* TT cross interpolation (Sec. 3.3): y ~ F where F is the entrywise function
 * `fn` of the input TTs, by alternating maximum-volume sweeps seeded by the
 * guess x0, kick fibres per sweep drawn from SplitMix64(seed), and a final
 * round at (tol, rank_cap).  fparams (host):
 *   TT_FN_ENTRY      : unused;
 *   TT_FN_WENO_S1    : {eps, side (-1: right-face value, +1: left-face value),
 *                       mode (0: stencil along the first index, 1: second)};
 *   TT_FN_WENO_S2    : {eps, mode (1: output n1 x 3*n2, columns m*n2+j;
 *                       0: output 3*n1 x n2, rows m*n1+i), nq (= 3)};
 *   TT_FN_LLF_LAMBDA : {g}; inputs = {h-, hu-, h+, hu+} (hu = hv for y faces).
 *   TT_FN_LLF_FLUX   : {g, direction (0: x faces, 1: y faces)}; inputs = {h-, hu-, hv-, h+, hu+, hv+},
 *                      each n1 x n2; y has 3 n1 rows: entry (c n1 + i, j) is component c of
 *                      F^(Q-, Q+) = (F(Q-) + F(Q+))/2 - lambda (Q+ - Q-)/2 at face point (i, j), with F the
 *                      nonlinear physical flux normal to the faces (Eq. nonlinear-SWE) and lambda the
 *                      larger |u_n| + sqrt(g h) of the two states.
 * The output shape is (y->n1, y->n2). */
size_t tt_cross_workspace_size(int32_t n1, int32_t n2, int32_t rank_in, int32_t rank_cap,
                               int32_t kick);
tt_status tt_cross(int32_t fn, const tt2* inputs, int32_t ninputs, const tt2* x0,
                   const double* fparams, double tol, int32_t rank_cap, int32_t kick,
                   int32_t max_sweeps, uint32_t seed, tt2* y, int32_t* sweeps_out, void* ws,
                   size_t ws_bytes, void* stream);

/* Maximum-volume rows (Sec. 3.3, the pivot choice of every cross sweep): r
 * row indices I of the n x r FP64 matrix U (device, column-major, ld n) such
 * that every entry of U U[I, :]^{-1} has magnitude at most 1 + delta.  Rows
 * are first chosen by partial pivoting, then swapped one at a time (the
 * largest entry above 1 + delta, ties to the smallest row-major index) until
 * none exceeds it or max_iter swaps were made (the bound may then not hold;
 * no error).  The choice compares magnitudes only and is made in FP32.
 * I: device int32[r], written.  Requires 1 <= r <= 128, n >= r. */
size_t tt_maxvol_workspace_size(int32_t n, int32_t r);
tt_status tt_maxvol(const double* U, int32_t n, int32_t r, double delta, int32_t max_iter, int32_t* I,
                    void* ws, size_t ws_bytes, void* stream);

/* Taylor-series TT reciprocal, Algorithm 1: y ~ 1/x with x_avg = sum(x)/N,
 * x~ = round(1 - x/x_avg), dy <- round(dy o x~), y <- round(y + dy) until
 * ||dy||_F / sqrt(N) <= tol.  TT_ERR_NOCONV after max_iter iterations. */
size_t tt_reciprocal_workspace_size(int32_t n1, int32_t n2, int32_t rank_in, int32_t rank_cap);
tt_status tt_reciprocal(const tt2* x, double tol, int32_t rank_cap, int32_t max_iter, tt2* y,
                        int32_t* iters_out, void* ws, size_t ws_bytes, void* stream);

/* Linear reconstruction on cores (Sec. 4.3.1) of one field for the faces
 * normal to `direction` (0: x faces, 1: y faces), scheme TT_UP3 | TT_UP5.
 * Outputs qm (state left of face: cell i-1's right-face value) and qp (cell
 * i's left-face value), rank = x.rank, stacked over the Gauss points:
 * x faces n1 x (nq n2), y faces (nq n1) x n2, quadrature index outermost. */
tt_status tt_recon_linear(const tt2* x, int32_t direction, int32_t scheme, tt2* qm, tt2* qp,
                          void* stream);

/* Library version string. */
const char* tt_fv_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TT_FV_H */
