// The TT finite-volume SSP-RK3 stage (Sec. 4) and the C ABI (include/tt_fv.h).
//
// Stage composition (Sec. 4.1-4.4):
//  * reconstruction: Upwind3/Upwind5 by stencils on one core at a time
//    (Sec. 4.3.1); WENO5 by two crosses per side (Algorithms 2 and 3), Step-2
//    results stored N x (Nq N) for x faces and (Nq N) x N for y faces with the
//    quadrature index outermost;
//  * LLF flux in TT (Eq. LLF-TT): linear SWE by TT sums with lambda =
//    sqrt(gH), no rounding; nonlinear SWE with 1/h by Algorithm 1, every
//    Hadamard product and sum rounded, lambda by cross;
//  * face quadrature, (T - 1)/dx on the core normal to the face, source term;
//  * F(u) = round(u + dt L(u)) and the SSP-RK3 combinations of Eq. tt-ssprk3.
// Face convention: face row i of an x-face TT is the face x_{i-1/2}; Qm holds
// cell i-1's right-face value, Qp cell i's left-face value.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <algorithm>
#include <chrono>

#include "coeffs.cuh"
#include "tt_ops.cuh"

namespace ttfv {

// ============================================================== helpers
static TT alloc_tt(Arena& ar, int n1, int n2, int cap) {
  TT t;
  t.n1 = n1;
  t.n2 = n2;
  t.cap = cap;
  t.r = 0;
  t.a = ar.get<double>((size_t)n1 * cap);
  t.b = ar.get<double>((size_t)n2 * cap);
  return t;
}

static void copy_tt(Exec& ex, const TT& src, TT& dst) {
  TT_REQUIRE(src.n1 == dst.n1 && src.n2 == dst.n2 && src.r <= dst.cap, TT_ERR_ARG);
  scaled_copy(ex, dst.a, src.a, (long)src.n1 * src.r, 1.0);
  scaled_copy(ex, dst.b, src.b, (long)src.n2 * src.r, 1.0);
  dst.r = src.r;
}

static TT const_tt(Exec& ex, int n1, int n2, double c) {
  TT t = alloc_tt(*ex.ar, n1, n2, 1);
  fill(ex, t.a, n1, c);
  fill(ex, t.b, n2, 1.0);
  t.r = 1;
  return t;
}

// ============================================================== Algorithm 1
// One reciprocal laid out as task-graph nodes.  The roundings are those of the
// serial loop, in its order per chain: xt = round(1 - x / x_avg), then for
// k = 1, 2, ...: dy <- round(dy o xt) and its norm (the stop test), y <-
// round(y + dy).  dy alternates between two buffers, so the y update of
// iteration k runs beside the dy rounding of iteration k + 1; the last node
// scales y by 1 / x_avg.
struct Reciprocal {
  TaskGraph* G = nullptr;
  const TT* x = nullptr;
  TT* y = nullptr;
  double tol = 0.0, x_avg = 1.0, err = 1.0;
  int cap = 0, max_iter = 0, prio = 0, it = 0;
  bool urgent = false;  // the chain is on the stage's critical path
  TT xt, dy[2];
  int reader[2] = {-1, -1};  // the y update that reads dy[b]
  int last_y = -1;
  int done = -1;
  bool noconv = false;
};

static void taylor_dy(Reciprocal& R, int k, int prev);

static void taylor_y(Reciprocal& R, int b, int dy_node) {
  const int yk = R.G->add(
      "taylor_y", R.prio,
      [&R, b](Exec& cx) { round_sum(cx, {Term{1.0, *R.y}, Term{1.0, R.dy[b]}}, R.tol, R.cap, *R.y); },
      {dy_node, R.last_y}, false, R.urgent);
  R.reader[b] = yk;
  R.last_y = yk;
}

// iteration k >= 1 writes dy[k & 1] from dy[(k - 1) & 1] (node prev); the
// buffer it overwrites was last read by the y update of iteration k - 2
static void taylor_dy(Reciprocal& R, int k, int prev) {
  const int b = k & 1;
  R.G->add(
      "taylor_dy", R.prio,
      [&R, k, b](Exec& cx) {
        const RoundInfo ri = round_hadamard(cx, R.dy[b ^ 1], R.xt, R.tol, R.cap, R.dy[b]);
        // ||dy||_F of the rounded product from its rounding: the kept part
        // of the truncated SVD, ||M||^2 - (discarded)^2 (the range finder's
        // residual is outside M), so the stop test needs no kernel or sync
        const double kept2 = ri.norm * ri.norm - (ri.err * ri.err - ri.resid * ri.resid);
        const double dy_norm = std::sqrt(std::max(kept2, 0.0));
        // the sizing pass runs two iterations: the second multiplies a dy of
        // full rank, the largest product of the loop
        R.err = cx.dry ? (k < 2 ? 1.0 : 0.0) : dy_norm / std::sqrt((double)R.x->n1 * R.x->n2);
        R.it = k;
        const int me = TaskGraph::self();
        taylor_y(R, b, me);
        if (R.err > R.tol && k < R.max_iter) {
          taylor_dy(R, k + 1, me);
        } else {
          R.G->depend(R.done, R.last_y);
          R.G->release(R.done);
        }
      },
      {prev, R.reader[b]}, false, R.urgent);
}

// Adds the nodes of y = 1/x (x and y preallocated; x's cores are read when
// the first node runs, after `after`).  Returns the node after which y holds
// the result; R must outlive G.run(), after which R.noconv and R.it hold the
// stop-test outcome and the iteration count.
static int reciprocal_nodes(TaskGraph& G, Exec& ex, const TT& x, double tol, int cap, int max_iter, TT& y,
                            int after, int prio, Reciprocal& R, bool urgent = false) {
  const int n1 = x.n1, n2 = x.n2;
  TT_REQUIRE(y.cap >= cap && y.n1 == n1 && y.n2 == n2, TT_ERR_ARG);
  R.G = &G;
  R.x = &x;
  R.y = &y;
  R.tol = effective_tol(ex, tol);  // a precision form stops at its own rounding level
  R.cap = cap;
  R.max_iter = max_iter;
  R.prio = prio;
  R.urgent = urgent;
  R.xt = alloc_tt(*ex.ar, n1, n2, cap);
  R.dy[0] = alloc_tt(*ex.ar, n1, n2, cap);
  R.dy[1] = alloc_tt(*ex.ar, n1, n2, cap);
  R.done = G.add(
      "taylor_scale", prio,
      [&R](Exec& cx) {
        cx.taylor_iters += R.it;
        scaled_copy(cx, R.y->a, R.y->a, (long)R.y->n1 * R.y->r, 1.0 / R.x_avg);
        R.noconv = R.err > R.tol;
      },
      {}, true, urgent);
  G.add(
      "taylor_init", prio,
      [&R](Exec& cx) {
        const TT& xx = *R.x;
        double* sn = cx.ar->get<double>(2);
        tt_sum_norm(cx, xx, sn);
        double v[2];
        fetch_doubles(cx, sn, 2, v);
        R.x_avg = cx.dry ? 1.0 : v[0] / ((double)xx.n1 * xx.n2);
        TT one = const_tt(cx, xx.n1, xx.n2, 1.0);
        round_sum(cx, {Term{1.0, one}, Term{-1.0 / R.x_avg, xx}}, R.tol, R.cap, R.xt);
        copy_tt(cx, one, R.dy[0]);
        copy_tt(cx, one, *R.y);
        const int me = TaskGraph::self();
        if (R.err > R.tol && R.max_iter > 0) {
          taylor_dy(R, 1, me);
        } else {
          R.G->depend(R.done, me);
          R.G->release(R.done);
        }
      },
      {after}, false, urgent);
  return R.done;
}

int reciprocal(Exec& ex, const TT& x, double tol, int cap, int max_iter, TT& y, bool* noconv) {
  Scope sc(*ex.ar);
  TaskGraph G(ex, 2);
  Reciprocal R;
  reciprocal_nodes(G, ex, x, tol, cap, max_iter, y, -1, 0, R);
  G.run();
  if (noconv) *noconv = R.noconv;
  return R.it;
}

// ============================================================== linear recon
// Non-periodic window: tap t reads input row i + base0 + t (no wrap; the
// caller guarantees the rows exist)
static void add_taps_window(StencilOut& o, const double* coef, int ntap, int base0) {
  for (int t = 0; t < ntap; ++t) {
    if (coef[t] == 0.0) continue;
    TT_REQUIRE(o.ntaps < kMaxTaps, TT_ERR_ARG);
    o.shift[o.ntaps] = 0;
    o.base[o.ntaps] = base0 + t;
    o.coef[o.ntaps] = coef[t];
    o.ntaps++;
  }
}

static void add_taps(StencilOut& o, const double* coef, int ntap, int shift0, int base) {
  for (int t = 0; t < ntap; ++t) {
    if (coef[t] == 0.0) continue;
    TT_REQUIRE(o.ntaps < kMaxTaps, TT_ERR_ARG);
    o.shift[o.ntaps] = shift0 + t;
    o.base[o.ntaps] = base;
    o.coef[o.ntaps] = coef[t];
    o.ntaps++;
  }
}

// Step 1 on the core normal to the faces (right-face stencil shifted by one
// cell for Qm, left-face stencil for Qp), Step 2 on the other core stacked
// over the Gauss points (Sec. 4.3.1).
void recon_linear(Exec& ex, const TT& x, int direction, int scheme, TT& qm, TT& qp) {
  const ReconCoeffs& R = recon_coeffs();
  const int nq = scheme == TT_UP3 ? 2 : 3;
  const double* right = scheme == TT_UP3 ? R.up3_minus : R.up5_minus;
  const double* left = scheme == TT_UP3 ? R.up3_plus : R.up5_plus;
  const double* nrm_core = direction == 0 ? x.a : x.b;
  const double* tan_core = direction == 0 ? x.b : x.a;
  const int nn = direction == 0 ? x.n1 : x.n2;  // normal mode size
  const int nt = direction == 0 ? x.n2 : x.n1;  // tangential mode size
  double* m_nrm = direction == 0 ? qm.a : qm.b;
  double* p_nrm = direction == 0 ? qp.a : qp.b;
  double* stack = direction == 0 ? qm.b : qm.a;
  StencilSet s1;
  s1.nout = 2;
  s1.out[0].dst = m_nrm;
  s1.out[0].ld = nn;
  add_taps(s1.out[0], right, 5, -2 - 1, 0);  // Qm[i] = right-face value of cell i-1
  s1.out[1].dst = p_nrm;
  s1.out[1].ld = nn;
  add_taps(s1.out[1], left, 5, -2, 0);
  stencil(ex, s1, nrm_core, nn, nn, x.r);
  StencilSet s2;
  s2.nout = nq;
  for (int m = 0; m < nq; ++m) {
    s2.out[m].dst = stack;
    s2.out[m].ld = (long)nq * nt;
    s2.out[m].row0 = m * nt;
    if (nq == 2)
      add_taps(s2.out[m], R.lin2[m], 3, -1, 0);
    else
      add_taps(s2.out[m], R.lin3[m], 5, -2, 0);
  }
  stencil(ex, s2, tan_core, nt, nt, x.r);
  // Qp shares the stacked core of Qm
  if (direction == 0)
    qp.b = qm.b;
  else
    qp.a = qm.a;
  qm.r = qp.r = x.r;
}

// ============================================================== solver context
struct Solver {
  tt_fv_params p{};
  cudaStream_t s = nullptr;
  Arena ar;
  Exec ex;
  TT Qn[3], Qs[3];
  int step_count = 0;
  int next_stage = 0;
  int nq = 2;
  int h_int[16];
  double h_dbl[16];
  Prof prof;
  StreamPool pool;
  double section_ms[6] = {};
  MlpNet net;                      // learned-pivot network (caller-owned weights)
  PivotRecorder* rec = nullptr;    // training-data capture, when enabled
  // converged column pivots of each cross site at its previous call:
  // WENO (direction, field, side, step) = 24 sites, then LLF lambda per direction
  // (then the LF-cross flux per direction)
  std::vector<int> sites[28];
  // range-finder sketch width that certified the previous lambda o jump
  // rounding of each (direction, component) within the current step
  int rf_hint[2][3] = {};
  // the previous stage's LLF lambda of each direction (nonlinear SWE) within
  // the current step: the initial guess of the next lambda cross
  TT lam_prev[2];
  bool lam_prev_ok[2] = {false, false};
  // tolerances of the current step (Sec. 4.4): p.tol holds eps_TT of the
  // rounds and crosses, tol_u[c] the per-field forward-Euler and SSP rounds
  double tol_u[3] = {0.0, 0.0, 0.0};
  // external source (tt_fv_set_forcing): plane waves, the time of the
  // current state and the time the current stage evaluates L at
  std::vector<tt_wave> waves;
  double time = 0.0, stage_time = 0.0;
  // exact solution on the x-boundary ghost cells (bc_x = TT_BC_EXACT)
  std::vector<tt_wave> bwaves;
  bool boundary_set = false;
  ~Solver();
};

// Captured (features, label) rows of the crosses of one solver
struct PivotRecorder {
  std::mutex mu;
  std::vector<float> X;  // rows x kMlpFeatures, row-major
  std::vector<float> y;
};

Solver::~Solver() {
  delete rec;
  for (cudaEvent_t e : prof.pool) cudaEventDestroy(e);
  for (const Prof::Rec& r : prof.pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
}

void record_pivots(Exec& ex, const TT& x0, const std::vector<int>& prev, const std::vector<int>& J) {
  if (ex.dry || !ex.pivot_rec) return;
  const int n2 = x0.n2;
  Scope sc(*ex.ar);
  float* X = ex.ar->get<float>((size_t)n2 * kMlpFeatures);
  mlp_features_host_prev(ex, x0, prev, X);
  std::vector<float> h((size_t)n2 * kMlpFeatures);
  TT_CUDA(cudaMemcpyAsync(h.data(), X, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, ex.s));
  host_wait(ex);
  ex.syncs++;
  std::vector<float> lab(n2, 0.0f);
  for (int j : J)
    if (j >= 0 && j < n2) lab[j] = 1.0f;
  PivotRecorder& R = *ex.pivot_rec;
  std::lock_guard<std::mutex> lk(R.mu);
  for (int j = 0; j < n2; ++j)
    for (int q = 0; q < kMlpFeatures; ++q) R.X.push_back(h[j + (size_t)q * n2]);
  R.y.insert(R.y.end(), lab.begin(), lab.end());
}

static int nq_of(int recon) { return recon == TT_UP3 ? 2 : 3; }

// ---------------------------------------------------------------- external source
struct WaveSet {
  int n;
  double amp[TT_MAX_WAVES], kx[TT_MAX_WAVES], ky[TT_MAX_WAVES], om[TT_MAX_WAVES], ph[TT_MAX_WAVES];
  double dk[TT_MAX_WAVES];  // decay in x (0: a plane wave)
};

__device__ __forceinline__ double sinc_dev(double z) { return z == 0.0 ? 1.0 : sin(z) / z; }

// Averages over the cell [i dx, (i + 1) dx] of exp(-dk x) cos(kx x) (cx) and
// exp(-dk x) sin(kx x) (sx): for dk = 0 the centre values times
// sinc(kx dx / 2); otherwise the real and imaginary parts of
// exp(w x_i) (exp(w dx) - 1) / (w dx), w = -dk + i kx, with exp(w dx) - 1
// formed from expm1 and a half-angle sine (no cancellation for small dx).
__device__ __forceinline__ void wave_x(double kx, double dk, int i, double dx, double& cx, double& sx) {
  if (dk == 0.0) {
    const double a = kx * (i + 0.5) * dx, s = sinc_dev(0.5 * kx * dx);
    cx = s * cos(a);
    sx = s * sin(a);
    return;
  }
  const double x1 = i * dx, e1 = exp(-dk * x1), c1 = cos(kx * x1), s1 = sin(kx * x1);
  const double hs = sin(0.5 * kx * dx);
  const double dr = expm1(-dk * dx) * cos(kx * dx) - 2.0 * hs * hs, di = exp(-dk * dx) * sin(kx * dx);
  const double pr = e1 * (c1 * dr - s1 * di), pim = e1 * (c1 * di + s1 * dr);
  const double m = 1.0 / ((dk * dk + kx * kx) * dx);
  cx = (-dk * pr + kx * pim) * m;
  sx = (-kx * pr - dk * pim) * m;
}

// Cell averages of sum_w amp_w cos(kx_w x + ky_w y - om_w t + ph_w) as a TT of
// rank 2 n: A[:, 2w] = sx cos(kx xc), A[:, 2w+1] = -sx sin(kx xc),
// B[:, 2w] = amp sy cos(ky yc - om t + ph), B[:, 2w+1] = amp sy sin(...), with
// sx = sinc(kx dx/2), sy = sinc(ky dy/2) (the exact average of a plane wave
// over a cell is its centre value times these factors).
__global__ void k_wave_cores(WaveSet w, double t, int n1, int n2, double dx, double dy, double* __restrict__ A,
                             double* __restrict__ B) {
  const long na = (long)n1 * 2 * w.n, total = na + (long)n2 * 2 * w.n;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
    if (q < na) {
      const int i = int(q % n1), col = int(q / n1), v = col >> 1;
      double cx, sx;
      wave_x(w.kx[v], w.dk[v], i, dx, cx, sx);
      A[q] = (col & 1) ? -sx : cx;
    } else {
      const long r = q - na;
      const int j = int(r % n2), col = int(r / n2), v = col >> 1;
      const double b = w.ky[v] * (j + 0.5) * dy - w.om[v] * t + w.ph[v];
      const double sy = w.amp[v] * sinc_dev(0.5 * w.ky[v] * dy);
      B[r] = (col & 1) ? sy * sin(b) : sy * cos(b);
    }
  }
}

// Number of source waves of field c (in the sizing pass: the most allowed).
static int wave_count(const Solver& S, const Exec& ex, int c) {
  if (ex.dry) return S.p.forcing_waves;
  int n = 0;
  for (const tt_wave& w : S.waves) n += w.field == c;
  return n;
}

// The source of field c at the current stage's time as a TT allocated from
// ex's arena (rank 2 per wave); false when the field has no wave.
static bool source_tt(Solver& S, Exec& ex, int c, TT& out) {
  const int nw = wave_count(S, ex, c);
  if (nw <= 0) return false;
  out = alloc_tt(*ex.ar, S.p.nx, S.p.ny, 2 * nw);
  out.r = 2 * nw;
  if (ex.dry) return true;
  WaveSet ws{};
  for (const tt_wave& w : S.waves)
    if (w.field == c) {
      ws.amp[ws.n] = w.amp;
      ws.kx[ws.n] = w.kx;
      ws.ky[ws.n] = w.ky;
      ws.om[ws.n] = w.omega;
      ws.ph[ws.n] = w.phase;
      ws.dk[ws.n] = w.decay;
      ws.n++;
    }
  const long total = (long)(S.p.nx + S.p.ny) * 2 * nw;
  const int blocks = std::max(1, std::min(ceil_div(total, 256), 1184));
  TT_KERNEL(ex, K_OTHER, 20.0 * total, 8.0 * total,
            k_wave_cores<<<blocks, 256, 0, ex.s>>>(ws, S.stage_time, S.p.nx, S.p.ny, S.p.lx / S.p.nx,
                                                   S.p.ly / S.p.ny, out.a, out.b));
  return true;
}

// Linear (Upwind3/Upwind5) faces of one field for direction d (0: x, 1: y)
static void faces_linear(Solver& S, Exec& ex, const TT& q, int d, TT& qm, TT& qp) {
  const int n1 = q.n1, n2 = q.n2, nq = S.nq;
  const int f1 = d == 0 ? n1 : nq * n1, f2 = d == 0 ? nq * n2 : n2;
  qm.n1 = qp.n1 = f1;
  qm.n2 = qp.n2 = f2;
  qm.cap = qp.cap = q.r;
  if (d == 0) {
    qm.a = ex.ar->get<double>((size_t)n1 * q.r);
    qp.a = ex.ar->get<double>((size_t)n1 * q.r);
    qm.b = ex.ar->get<double>((size_t)f2 * q.r);
  } else {
    qm.b = ex.ar->get<double>((size_t)n2 * q.r);
    qp.b = ex.ar->get<double>((size_t)n2 * q.r);
    qm.a = ex.ar->get<double>((size_t)f1 * q.r);
  }
  recon_linear(ex, q, d, S.p.recon, qm, qp);
}

// ---------------------------------------------------------------- bounded x
constexpr int kGhost = 3;  // cells beyond each x boundary that one stage's stencils read

// The TT of a field with kGhost ghost rows beyond each x boundary holding the
// exact solution's cell averages at time t (Sec. 5.1 / 5.3 boundary values):
// first core Ae ((nx + 2 kGhost) x (r + 2 n)): the field's columns on the real
// rows and zero on the ghost rows, then the waves' rank-2 columns on the ghost
// rows and zero on the real rows; second core Be (ny x (r + 2 n)): the
// field's second core, then the waves' y factors (as in k_wave_cores).
__global__ void k_extend_x(const double* __restrict__ A, const double* __restrict__ B, int nx, int ny, int r,
                           WaveSet w, double t, double dx, double dy, double* __restrict__ Ae,
                           double* __restrict__ Be) {
  const int ne = nx + 2 * kGhost, R = r + 2 * w.n;
  const long na = (long)ne * R, total = na + (long)ny * R;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
    if (q < na) {
      const int i = int(q % ne), col = int(q / ne);
      const bool ghost = i < kGhost || i >= kGhost + nx;
      double v = 0.0;
      if (col < r) {
        if (!ghost) v = A[(i - kGhost) + (size_t)col * nx];
      } else if (ghost) {
        const int wc = col - r, wv = wc >> 1;
        double cx, sx;
        wave_x(w.kx[wv], w.dk[wv], i - kGhost, dx, cx, sx);
        v = (wc & 1) ? -sx : cx;
      }
      Ae[q] = v;
    } else {
      const long rr = q - na;
      const int j = int(rr % ny), col = int(rr / ny);
      double v;
      if (col < r) {
        v = B[j + (size_t)col * ny];
      } else {
        const int wc = col - r, wv = wc >> 1;
        const double b = w.ky[wv] * (j + 0.5) * dy - w.om[wv] * t + w.ph[wv];
        const double sy = w.amp[wv] * sinc_dev(0.5 * w.ky[wv] * dy);
        v = (wc & 1) ? sy * sin(b) : sy * cos(b);
      }
      Be[rr] = v;
    }
  }
}

// Field c's TT extended by the boundary ghost rows at the current stage's time
static TT extend_x(Solver& S, Exec& ex, const TT& q, int c) {
  int nw = 0;
  WaveSet ws{};
  if (ex.dry) {
    nw = S.p.boundary_waves;
  } else {
    for (const tt_wave& w : S.bwaves)
      if (w.field == c) {
        ws.amp[ws.n] = w.amp;
        ws.kx[ws.n] = w.kx;
        ws.ky[ws.n] = w.ky;
        ws.om[ws.n] = w.omega;
        ws.ph[ws.n] = w.phase;
        ws.dk[ws.n] = w.decay;
        ws.n++;
      }
    nw = ws.n;
  }
  const int nx = S.p.nx, ny = S.p.ny, ne = nx + 2 * kGhost, R = q.r + 2 * nw;
  TT e = alloc_tt(*ex.ar, ne, ny, R);
  e.r = R;
  if (ex.dry) return e;
  const long total = (long)(ne + ny) * R;
  const int blocks = std::max(1, std::min(ceil_div(total, 256), 1184));
  TT_KERNEL(ex, K_OTHER, 20.0 * (ne + ny) * 2.0 * nw, 8.0 * (double)total + 8.0 * (nx + ny) * (double)q.r,
            k_extend_x<<<blocks, 256, 0, ex.s>>>(q.a, q.b, nx, ny, q.r, ws, S.stage_time, S.p.lx / nx,
                                                 S.p.ly / ny, e.a, e.b));
  return e;
}

// Linear faces (Upwind3 / Upwind5) of a field from its extended TT e on the
// domain bounded in x: x faces are the nx + 1 faces x_{-1/2} .. x_{nx-1/2}
// (Qm: the right-face value of the cell below, ghost or real, Qp: the
// left-face value of the cell above), y faces those of the nx real rows
// with Step 2 in x reading the ghost rows; y stays periodic.
static void faces_linear_bounded(Solver& S, Exec& ex, const TT& e, int d, TT& qm, TT& qp) {
  const ReconCoeffs& Rc = recon_coeffs();
  const int nx = S.p.nx, ny = S.p.ny, nq = S.nq, ne = e.n1, R = e.r;
  const double* right = S.p.recon == TT_UP3 ? Rc.up3_minus : Rc.up5_minus;
  const double* left = S.p.recon == TT_UP3 ? Rc.up3_plus : Rc.up5_plus;
  const int f1 = d == 0 ? nx + 1 : nq * nx, f2 = d == 0 ? nq * ny : ny;
  qm.n1 = qp.n1 = f1;
  qm.n2 = qp.n2 = f2;
  qm.cap = qp.cap = R;
  if (d == 0) {
    qm.a = ex.ar->get<double>((size_t)f1 * R);
    qp.a = ex.ar->get<double>((size_t)f1 * R);
    qm.b = ex.ar->get<double>((size_t)f2 * R);
    qp.b = qm.b;
    // Step 1 in x without wrap: face k reads ghost-extended rows k .. k + 4
    // (Qm, cell k - 1) and k + 1 .. k + 5 (Qp, cell k)
    StencilSet s1;
    s1.nout = 2;
    s1.out[0].dst = qm.a;
    s1.out[0].ld = f1;
    add_taps_window(s1.out[0], right, 5, 0);
    s1.out[1].dst = qp.a;
    s1.out[1].ld = f1;
    add_taps_window(s1.out[1], left, 5, 1);
    stencil(ex, s1, e.a, ne, f1, R);
    StencilSet s2;  // Step 2 in y (periodic)
    s2.nout = nq;
    for (int m = 0; m < nq; ++m) {
      s2.out[m].dst = qm.b;
      s2.out[m].ld = (long)nq * ny;
      s2.out[m].row0 = m * ny;
      if (nq == 2)
        add_taps(s2.out[m], Rc.lin2[m], 3, -1, 0);
      else
        add_taps(s2.out[m], Rc.lin3[m], 5, -2, 0);
    }
    stencil(ex, s2, e.b, ny, ny, R);
  } else {
    qm.b = ex.ar->get<double>((size_t)ny * R);
    qp.b = ex.ar->get<double>((size_t)ny * R);
    qm.a = ex.ar->get<double>((size_t)f1 * R);
    qp.a = qm.a;
    StencilSet s1;  // Step 1 in y (periodic)
    s1.nout = 2;
    s1.out[0].dst = qm.b;
    s1.out[0].ld = ny;
    add_taps(s1.out[0], right, 5, -2 - 1, 0);
    s1.out[1].dst = qp.b;
    s1.out[1].ld = ny;
    add_taps(s1.out[1], left, 5, -2, 0);
    stencil(ex, s1, e.b, ny, ny, R);
    StencilSet s2;  // Step 2 in x at the Gauss points, real rows, no wrap
    s2.nout = nq;
    for (int m = 0; m < nq; ++m) {
      s2.out[m].dst = qm.a;
      s2.out[m].ld = (long)nq * nx;
      s2.out[m].row0 = m * nx;
      if (nq == 2)
        add_taps_window(s2.out[m], Rc.lin2[m], 3, kGhost - 1);
      else
        add_taps_window(s2.out[m], Rc.lin3[m], 5, kGhost - 2);
    }
    stencil(ex, s2, e.a, ne, nx, R);
  }
  qm.r = qp.r = R;
}

// One side of the WENO5 faces of one field (Algorithms 2 and 3): Step 1 by
// cross along the face normal, Step 2 by cross at all Gauss points; the
// "-" side (k = 0) is then shifted by one cell along the normal (Qm).
static void weno_side(Solver& S, Exec& ex, const TT& q, int d, int fieldc, int k, unsigned seed, TT& dst) {
  const tt_fv_params& p = S.p;
  const int n1 = q.n1, n2 = q.n2, cap = p.rank_cap;
  const int f1 = d == 0 ? n1 : 3 * n1, f2 = d == 0 ? 3 * n2 : n2;
  const double dx = p.lx / p.nx, dy = p.ly / p.ny;
  const double e1 = d == 0 ? dx * dx : dy * dy, e2 = d == 0 ? dy * dy : dx * dx;
  const int kick = p.kick > 0 ? p.kick : 4, sweeps = p.max_sweeps > 0 ? p.max_sweeps : 10;
  const unsigned seed_base = seed + 64u * d + 8u * fieldc;
  Scope sc(*ex.ar);
  const int site = ((d * 3 + fieldc) * 2 + k) * 2;
  CrossFn f1n;
  f1n.fn = TT_FN_WENO_S1;
  f1n.in = &q;
  f1n.nin = 1;
  f1n.site = &S.sites[site];
  f1n.prm[0] = e1;
  f1n.prm[1] = k == 0 ? -1.0 : 1.0;
  f1n.prm[2] = d;
  TT vt = alloc_tt(*ex.ar, n1, n2, cap);
  cross(ex, f1n, n1, n2, q, p.tol, cap, kick, sweeps, seed_base + 4u * k, vt);
  // initial guess of Step 2: the Step-1 result repeated over the Gauss points
  TT x0 = d == 0 ? alloc_tt(*ex.ar, n1, 3 * n2, vt.r) : alloc_tt(*ex.ar, 3 * n1, n2, vt.r);
  x0.r = vt.r;
  if (d == 0) {
    scaled_copy(ex, x0.a, vt.a, (long)n1 * vt.r, 1.0);
    repeat_rows(ex, x0.b, vt.b, n2, vt.r, 3);
  } else {
    scaled_copy(ex, x0.b, vt.b, (long)n2 * vt.r, 1.0);
    repeat_rows(ex, x0.a, vt.a, n1, vt.r, 3);
  }
  CrossFn f2n;
  f2n.fn = TT_FN_WENO_S2;
  f2n.in = &vt;
  f2n.nin = 1;
  f2n.site = &S.sites[site + 1];
  f2n.prm[0] = e2;
  f2n.prm[1] = d == 0 ? 1.0 : 0.0;
  f2n.prm[2] = 3;
  TT tmp = alloc_tt(*ex.ar, f1, f2, cap);
  cross(ex, f2n, f1, f2, x0, p.tol, cap, kick, sweeps, seed_base + 4u * k + 1u, tmp);
  if (k == 0) {
    StencilSet st;
    st.nout = 1;
    double one = 1.0;
    if (d == 0) {
      st.out[0].dst = dst.a;
      st.out[0].ld = f1;
      add_taps(st.out[0], &one, 1, -1, 0);
      stencil(ex, st, tmp.a, f1, f1, tmp.r);
      scaled_copy(ex, dst.b, tmp.b, (long)f2 * tmp.r, 1.0);
    } else {
      st.out[0].dst = dst.b;
      st.out[0].ld = f2;
      add_taps(st.out[0], &one, 1, -1, 0);
      stencil(ex, st, tmp.b, f2, f2, tmp.r);
      scaled_copy(ex, dst.a, tmp.a, (long)f1 * tmp.r, 1.0);
    }
    dst.r = tmp.r;
  } else {
    copy_tt(ex, tmp, dst);
  }
}

// LLF flux of the linear SWE (TT sums only)
static void flux_linear(Solver& S, const TT qm[3], const TT qp[3], int d, std::vector<Term> out[3]) {
  const double g = S.p.g, H = S.p.H, lam = std::sqrt(g * H);
  const int k = d == 0 ? 1 : 2;
  for (int c = 0; c < 3; ++c) {
    out[c].clear();
    if (c == 0) {
      out[c].push_back(Term{0.5 * H, qm[k]});
      out[c].push_back(Term{0.5 * H, qp[k]});
    } else if (c == k) {
      out[c].push_back(Term{0.5 * g, qm[0]});
      out[c].push_back(Term{0.5 * g, qp[0]});
    }
    out[c].push_back(Term{-0.5 * lam, qp[c]});
    out[c].push_back(Term{0.5 * lam, qm[c]});
  }
}

// Nonlinear physical flux of one face side (Sec. 4.2): 1/h by Algorithm 1,
// u = round(hu o 1/h), v = round(hv o 1/h), then F = (hu, round(round(hu o u)
// + g/2 round(h o h)), round(hu o v)) for x faces and G = (hv, round(hv o u),
// round(round(hv o v) + g/2 round(h o h))) for y faces.  F[0] is left to the caller.
// lambda = max(|u-| + sqrt(g h-), |u+| + sqrt(g h+)) on the faces by cross,
// from the initial guess x0 (the paper leaves it open: h+ at the first
// stage, then the previous stage's lambda of the same direction)
static void face_lambda(Solver& S, Exec& ex, const TT qm[3], const TT qp[3], int d, unsigned seed, const TT& x0,
                        TT& lam) {
  const tt_fv_params& p = S.p;
  const int k = d == 0 ? 1 : 2;
  TT ins[4] = {qm[0], qm[k], qp[0], qp[k]};
  CrossFn fl;
  fl.fn = TT_FN_LLF_LAMBDA;
  fl.in = ins;
  fl.nin = 4;
  fl.site = &S.sites[24 + d];
  fl.prm[0] = p.g;
  const int kick = p.kick > 0 ? p.kick : 4, sweeps = p.max_sweeps > 0 ? p.max_sweeps : 10;
  cross(ex, fl, qm[0].n1, qm[0].n2, x0, p.tol, p.rank_cap, kick, sweeps, seed, lam);
}

// LF-cross (Sec. 4.2, the alternative the paper weighs against the product
// form): the LLF flux vector of direction d at the faces, F^(Q-, Q+) =
// (F(Q-) + F(Q+))/2 - lambda (Q+ - Q-)/2, by one cross of the six face states
// with its three components stacked along the first mode, then split into
// one TT per component (rows c f1 .. (c+1) f1 of the first core, the second
// core shared).  Initial guess: the h- faces (their column mode is the
// flux's); the cross ends in a round at tol like every cross.
static void flux_by_cross(Solver& S, Exec& ex, const TT qm[3], const TT qp[3], int d, unsigned seed, TT Fh[3]) {
  const tt_fv_params& p = S.p;
  const int f1 = qm[0].n1, f2 = qm[0].n2, cap = p.rank_cap;
  Scope sc(*ex.ar);
  TT ins[6] = {qm[0], qm[1], qm[2], qp[0], qp[1], qp[2]};
  CrossFn fl;
  fl.fn = TT_FN_LLF_FLUX;
  fl.in = ins;
  fl.nin = 6;
  fl.site = &S.sites[26 + d];
  fl.prm[0] = p.g;
  fl.prm[1] = d;
  const int kick = p.kick > 0 ? p.kick : 4, sweeps = p.max_sweeps > 0 ? p.max_sweeps : 10;
  TT st = alloc_tt(*ex.ar, 3 * f1, f2, cap);
  cross(ex, fl, 3 * f1, f2, qm[0], p.tol, cap, kick, sweeps, seed, st);
  StencilSet ss;
  ss.nout = 3;
  const double one = 1.0;
  for (int c = 0; c < 3; ++c) {
    TT_REQUIRE(Fh[c].n1 == f1 && Fh[c].n2 == f2 && Fh[c].cap >= st.r, TT_ERR_ARG);
    ss.out[c].dst = Fh[c].a;
    ss.out[c].ld = f1;
    add_taps(ss.out[c], &one, 1, 0, c * f1);
  }
  stencil(ex, ss, st.a, 3L * f1, f1, st.r);
  for (int c = 0; c < 3; ++c) {
    scaled_copy(ex, Fh[c].b, st.b, (long)f2 * st.r, 1.0);
    Fh[c].r = st.r;
  }
}

// LLF combination of one component (Eq. LLF-TT): with dd = round(Q+ - Q-) and
// ld = round(lambda o dd) computed earlier, out = round(F-/2 + F+/2 - ld/2)
static void llf_combine(Solver& S, Exec& ex, const TT& Fm, const TT& Fp, const TT& ld, TT& out) {
  round_sum(ex, {Term{0.5, Fm}, Term{0.5, Fp}, Term{-0.5, ld}}, S.p.tol, S.p.rank_cap, out);
}

// sum_m w_m over the stacked index, then (T - 1)/h on the normal core:
// out = the TT of (F_{i+1/2} - F_{i-1/2}) / h (Eq. SWE-system-TT); out is an
// nx x ny TT with room for Fh's rank.
static void quad_and_difference(Solver& S, Exec& ex, const TT& Fh, int d, TT& out) {
  const ReconCoeffs& R = recon_coeffs();
  const int nq = S.nq;
  const double* w = nq == 2 ? R.w2 : R.w3;
  const int n = d == 0 ? S.p.ny : S.p.nx;  // tangential size
  const int nn = d == 0 ? S.p.nx : S.p.ny;
  const double h = d == 0 ? S.p.lx / S.p.nx : S.p.ly / S.p.ny;
  TT_REQUIRE(out.n1 == S.p.nx && out.n2 == S.p.ny && out.cap >= Fh.r, TT_ERR_ARG);
  out.r = Fh.r;
  StencilSet sq;
  sq.nout = 1;
  sq.out[0].dst = d == 0 ? out.b : out.a;
  sq.out[0].ld = n;
  for (int m = 0; m < nq; ++m) {
    double c = w[m];
    add_taps(sq.out[0], &c, 1, 0, m * n);
  }
  stencil(ex, sq, d == 0 ? Fh.b : Fh.a, (long)nq * n, n, Fh.r);
  StencilSet sd;
  sd.nout = 1;
  sd.out[0].dst = d == 0 ? out.a : out.b;
  sd.out[0].ld = nn;
  const double cd[2] = {-1.0 / h, 1.0 / h};
  if (d == 0 && S.p.bc_x == TT_BC_EXACT) {
    // nx + 1 faces, difference without wrap
    TT_REQUIRE(Fh.n1 == nn + 1, TT_ERR_ARG);
    add_taps_window(sd.out[0], cd, 2, 0);
    stencil(ex, sd, Fh.a, nn + 1, nn, Fh.r);
    return;
  }
  add_taps(sd.out[0], cd, 2, 0, 0);
  stencil(ex, sd, d == 0 ? Fh.a : Fh.b, nn, nn, Fh.r);
}

struct SectionTimer {
  double& acc;
  std::chrono::steady_clock::time_point t0;
  explicit SectionTimer(double& a) : acc(a), t0(std::chrono::steady_clock::now()) {}
  ~SectionTimer() {
    acc += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

// Host threads (each with a stream and an arena slice) of a stage graph:
// TT_STAGE_WORKERS, else 16 -- the widest front of the nonlinear graph.
static int stage_workers() {
  static const int w = [] {
    const char* e = std::getenv("TT_STAGE_WORKERS");
    const int v = e ? std::atoi(e) : 0;
    return v >= 1 && v <= 48 ? v : 16;
  }();
  return w;
}

// F(u) = round(u + dt L(u)) for the three fields of the linear SWE
// (Eq. tt-forward-euler): faces (the 12 WENO crosses run as concurrent tasks),
// the LLF flux as TT sums, the quadrature and difference, the 3 final rounds.
static void forward_euler_linear(Solver& S, Exec& ex, const TT Q[3], unsigned seed, TT out[3]) {
  Scope sc(*ex.ar);
  const tt_fv_params& p = S.p;
  const int cap = p.rank_cap;
  std::vector<Term> terms[3];
  for (int c = 0; c < 3; ++c) terms[c].push_back(Term{1.0, Q[c]});
  TT qm[2][3], qp[2][3];
  int f1[2], f2[2];
  const bool bounded = p.bc_x == TT_BC_EXACT;
  for (int d = 0; d < 2; ++d) {
    f1[d] = d == 0 ? p.nx + (bounded ? 1 : 0) : S.nq * p.nx;
    f2[d] = d == 0 ? S.nq * p.ny : p.ny;
  }
  {
    SectionTimer st0(S.section_ms[0]);
    if (bounded) {
      for (int c = 0; c < 3; ++c) {
        const TT e = extend_x(S, ex, Q[c], c);
        for (int d = 0; d < 2; ++d) faces_linear_bounded(S, ex, e, d, qm[d][c], qp[d][c]);
      }
    } else if (p.recon == TT_WENO5) {
      for (int d = 0; d < 2; ++d)
        for (int c = 0; c < 3; ++c) {
          qm[d][c] = alloc_tt(*ex.ar, f1[d], f2[d], cap);
          qp[d][c] = alloc_tt(*ex.ar, f1[d], f2[d], cap);
        }
      parallel_tasks(ex, 12, [&](Exec& cx, int t) {
        const int d = t / 6, c = (t / 2) % 3, k = t % 2;
        weno_side(S, cx, Q[c], d, c, k, seed, k == 0 ? qm[d][c] : qp[d][c]);
      });
    } else {
      for (int d = 0; d < 2; ++d)
        for (int c = 0; c < 3; ++c) faces_linear(S, ex, Q[c], d, qm[d][c], qp[d][c]);
    }
  }
  {
    SectionTimer st3(S.section_ms[3]);
    for (int d = 0; d < 2; ++d) {
      std::vector<Term> fl[3];
      flux_linear(S, qm[d], qp[d], d, fl);
      for (int c = 0; c < 3; ++c) {
        const int R = total_rank(fl[c]);
        TT cat = alloc_tt(*ex.ar, f1[d], f2[d], R);
        tt_concat(ex, fl[c], cat);
        TT D = alloc_tt(*ex.ar, p.nx, p.ny, R);
        quad_and_difference(S, ex, cat, d, D);
        terms[c].push_back(Term{-p.dt, D});
      }
    }
  }
  if (p.f != 0.0) {
    terms[1].push_back(Term{p.dt * p.f, Q[2]});
    terms[2].push_back(Term{-p.dt * p.f, Q[1]});
  }
  for (int c = 0; c < 3; ++c) {
    TT src;
    if (source_tt(S, ex, c, src)) terms[c].push_back(Term{p.dt, src});
  }
  SectionTimer st4(S.section_ms[4]);
  parallel_tasks(ex, 3, [&](Exec& cx, int c) { round_sum(cx, terms[c], S.tol_u[c], cap, out[c]); });
}

// F(u) = round(u + dt L(u)) for the nonlinear SWE as one task graph.  Every
// cross, rounding and reciprocal of Sec. 4.2 and Eq. LLF-TT is a node that
// starts once its inputs exist: per face side, 1/h by Algorithm 1 (its two
// chains pipelined), u = round(hu o 1/h), v = round(hv o 1/h), h o h and the
// flux components; per direction the lambda cross; per component the LLF jump
// dd = round(Q+ - Q-), round(lambda o dd), the LLF combination and the
// quadrature/difference; per field the final round.  A node waits only for
// what it reads, so the reciprocal of one side starts when that side's h
// faces exist while other fields' faces are still being reconstructed.  Each
// quantity is the same sequence of roundings as in a serial evaluation.
static void forward_euler_graph(Solver& S, Exec& ex, const TT Q[3], unsigned seed, TT out[3]) {
  Scope sc(*ex.ar);
  const tt_fv_params& p = S.p;
  const int cap = p.rank_cap;
  const double tol = p.tol, g = p.g;
  const int mi = p.max_iter > 0 ? p.max_iter : 50;
  int f1[2], f2[2];
  for (int d = 0; d < 2; ++d) {
    f1[d] = d == 0 ? p.nx : S.nq * p.nx;
    f2[d] = d == 0 ? S.nq * p.ny : p.ny;
  }
  // phase milestones (ms from the start): the last face, flux, LLF,
  // quadrature and final-round node to finish
  const auto t_start = std::chrono::steady_clock::now();
  std::mutex mmu;
  double last[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  auto mark = [&](int phase) {
    const double t =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    std::lock_guard<std::mutex> lk(mmu);
    last[phase] = std::max(last[phase], t);
  };
  TaskGraph G(ex, stage_workers());
  TT qm[2][3], qp[2][3];
  int face[2][3][2];
  for (int d = 0; d < 2; ++d)
    for (int c = 0; c < 3; ++c) face[d][c][0] = face[d][c][1] = -1;
  if (p.recon == TT_WENO5) {
    for (int d = 0; d < 2; ++d)
      for (int c = 0; c < 3; ++c) {
        qm[d][c] = alloc_tt(*ex.ar, f1[d], f2[d], cap);
        qp[d][c] = alloc_tt(*ex.ar, f1[d], f2[d], cap);
      }
    for (int d = 0; d < 2; ++d)
      for (int c = 0; c < 3; ++c)
        for (int k = 0; k < 2; ++k)
          face[d][c][k] = G.add("weno_face", c == 0 ? 100 : 90, [&, d, c, k](Exec& cx) {
            weno_side(S, cx, Q[c], d, c, k, seed, k == 0 ? qm[d][c] : qp[d][c]);
            mark(0);
          }, {}, false, c == 0);
  } else {
    for (int d = 0; d < 2; ++d)
      for (int c = 0; c < 3; ++c) faces_linear(S, ex, Q[c], d, qm[d][c], qp[d][c]);
    mark(0);
  }
  TT F[2][2][3], lam[2], Fh[2][3], dd[2][3], ld[2][3], D[2][3];
  TT rh[2][2], hh[2][2], uu[2][2], vv[2][2];
  Reciprocal R[2][2];
  int qd_node[2][3];
  if (p.flux == TT_FLUX_CROSS) {
    // LF-cross: per direction one cross of the whole flux vector, then the
    // quadrature / difference of each component
    for (int d = 0; d < 2; ++d) {
      for (int c = 0; c < 3; ++c) {
        Fh[d][c] = alloc_tt(*ex.ar, f1[d], f2[d], cap);
        D[d][c] = alloc_tt(*ex.ar, p.nx, p.ny, cap);
      }
      std::vector<int> deps;
      for (int c = 0; c < 3; ++c)
        for (int k = 0; k < 2; ++k) deps.push_back(face[d][c][k]);
      const int fx = G.add("llf_flux_cross", 85, [&, d](Exec& cx) {
        flux_by_cross(S, cx, qm[d], qp[d], d, seed + 64u * d + 44u, Fh[d]);
        mark(2);
      }, deps, false, true);
      for (int c = 0; c < 3; ++c)
        qd_node[d][c] = G.add("quad_difference", 40, [&, d, c](Exec& cx) {
          quad_and_difference(S, cx, Fh[d][c], d, D[d][c]);
          mark(3);
        }, {fx}, false, true);
    }
  } else {
  for (int d = 0; d < 2; ++d) {
    lam[d] = alloc_tt(*ex.ar, f1[d], f2[d], cap);
    for (int sd = 0; sd < 2; ++sd) {
      for (int c = 1; c < 3; ++c) F[d][sd][c] = alloc_tt(*ex.ar, f1[d], f2[d], cap);
      rh[d][sd] = alloc_tt(*ex.ar, f1[d], f2[d], cap);
      hh[d][sd] = alloc_tt(*ex.ar, f1[d], f2[d], cap);
      uu[d][sd] = alloc_tt(*ex.ar, f1[d], f2[d], cap);
      vv[d][sd] = alloc_tt(*ex.ar, f1[d], f2[d], cap);
    }
    for (int c = 0; c < 3; ++c) {
      Fh[d][c] = alloc_tt(*ex.ar, f1[d], f2[d], cap);
      dd[d][c] = alloc_tt(*ex.ar, f1[d], f2[d], cap);
      ld[d][c] = alloc_tt(*ex.ar, f1[d], f2[d], cap);
      D[d][c] = alloc_tt(*ex.ar, p.nx, p.ny, cap);
    }
  }
  auto side = [&](int d, int sd) -> const TT* { return sd == 0 ? qm[d] : qp[d]; };
  int hh_node[2][2], vel_node[2][2][2], flux_node[2][2][3], lam_node[2], ld_node[2][3];
  for (int d = 0; d < 2; ++d) {
    const int k = d == 0 ? 1 : 2;  // the normal momentum hu (x) or hv (y)
    for (int sd = 0; sd < 2; ++sd) {
      const int rdone = reciprocal_nodes(G, ex, side(d, sd)[0], tol, cap, mi, rh[d][sd], face[d][0][sd], 80,
                                         R[d][sd], true);
      hh_node[d][sd] = G.add("h_o_h", 60, [&, d, sd](Exec& cx) {
        round_hadamard(cx, side(d, sd)[0], side(d, sd)[0], tol, cap, hh[d][sd]);
        mark(1);
      }, {face[d][0][sd]});
      for (int comp = 0; comp < 2; ++comp)
        vel_node[d][sd][comp] = G.add("velocity", 75, [&, d, sd, comp](Exec& cx) {
          round_hadamard(cx, side(d, sd)[1 + comp], rh[d][sd], tol, cap, comp == 0 ? uu[d][sd] : vv[d][sd]);
          mark(1);
        }, {rdone, face[d][1 + comp][sd]}, false, true);
      flux_node[d][sd][0] = -1;
      for (int comp = 1; comp < 3; ++comp)
        flux_node[d][sd][comp] = G.add("flux", 70, [&, d, sd, comp, k](Exec& cx) {
          const TT& qn = side(d, sd)[k];
          const TT& vel = comp == 1 ? uu[d][sd] : vv[d][sd];
          if (comp == k) {  // normal component: q_n o u_n + g h^2 / 2
            Scope s2(*cx.ar);
            TT t1 = alloc_tt(*cx.ar, f1[d], f2[d], cap);
            round_hadamard(cx, qn, vel, tol, cap, t1);
            round_sum(cx, {Term{1.0, t1}, Term{0.5 * g, hh[d][sd]}}, tol, cap, F[d][sd][comp]);
          } else {
            round_hadamard(cx, qn, vel, tol, cap, F[d][sd][comp]);
          }
          mark(1);
        }, {vel_node[d][sd][comp - 1], face[d][k][sd], comp == k ? hh_node[d][sd] : -1}, false, true);
    }
    lam_node[d] = G.add("llf_lambda", 85, [&, d](Exec& cx) {
      // lambda moves little from one stage to the next: the previous
      // stage's lambda is the initial guess (its pivots sit on the kinks
      // of the max), started by maxvol on it also in the learned form,
      // whose network was trained on h+ guesses (it proposes the first
      // stage's lambda pivots and every WENO face's)
      const bool warm = S.lam_prev_ok[d];
      const MlpNet* net = cx.pivot_net;
      if (warm) cx.pivot_net = nullptr;
      try {
        face_lambda(S, cx, qm[d], qp[d], d, seed + 64u * d + 40u, warm ? S.lam_prev[d] : qp[d][0], lam[d]);
      } catch (...) {
        cx.pivot_net = net;
        throw;
      }
      cx.pivot_net = net;
      if (!cx.dry) {
        copy_tt(cx, lam[d], S.lam_prev[d]);
        S.lam_prev_ok[d] = true;
      }
      mark(1);
    }, {face[d][0][0], face[d][0][1], face[d][k][0], face[d][k][1]});
    for (int c = 0; c < 3; ++c) {
      const int dd_node = G.add("llf_jump", 50, [&, d, c](Exec& cx) {
        round_sum(cx, {Term{1.0, qp[d][c]}, Term{-1.0, qm[d][c]}}, tol, cap, dd[d][c]);
        mark(1);
      }, {face[d][c][0], face[d][c][1]});
      ld_node[d][c] = G.add("lambda_o_jump", 55, [&, d, c](Exec& cx) {
        // the product of a non-smooth lambda and a jump keeps a wide numerical
        // rank: its sketch starts at the width that certified last time
        cx.rf_hint = &S.rf_hint[d][c];
        try {
          round_hadamard(cx, lam[d], dd[d][c], tol, cap, ld[d][c]);
        } catch (...) {
          cx.rf_hint = nullptr;
          throw;
        }
        cx.rf_hint = nullptr;
        mark(1);
      }, {lam_node[d], dd_node});
    }
    for (int c = 0; c < 3; ++c) {
      // the mass flux is the normal momentum itself
      std::vector<int> deps = c == 0 ? std::vector<int>{face[d][k][0], face[d][k][1]}
                                     : std::vector<int>{flux_node[d][0][c], flux_node[d][1][c]};
      deps.push_back(ld_node[d][c]);
      const int llf = G.add("llf_combine", 40, [&, d, c, k](Exec& cx) {
        llf_combine(S, cx, c == 0 ? qm[d][k] : F[d][0][c], c == 0 ? qp[d][k] : F[d][1][c], ld[d][c], Fh[d][c]);
        mark(2);
      }, deps, false, true);
      qd_node[d][c] = G.add("quad_difference", 40, [&, d, c](Exec& cx) {
        quad_and_difference(S, cx, Fh[d][c], d, D[d][c]);
        mark(3);
      }, {llf}, false, true);
    }
  }
  }  // products form
  for (int c = 0; c < 3; ++c)
    G.add("forward_euler", 30, [&, c](Exec& cx) {
      std::vector<Term> terms{Term{1.0, Q[c]}, Term{-p.dt, D[0][c]}, Term{-p.dt, D[1][c]}};
      if (p.f != 0.0 && c == 1) terms.push_back(Term{p.dt * p.f, Q[2]});
      if (p.f != 0.0 && c == 2) terms.push_back(Term{-p.dt * p.f, Q[1]});
      Scope s2(*cx.ar);
      TT src;
      if (source_tt(S, cx, c, src)) terms.push_back(Term{p.dt, src});
      round_sum(cx, terms, S.tol_u[c], cap, out[c]);
      mark(4);
    }, {qd_node[0][c], qd_node[1][c]}, false, true);
  G.run();
  for (int d = 0; d < 2; ++d)
    for (int sd = 0; sd < 2; ++sd) TT_REQUIRE(!R[d][sd].noconv, TT_ERR_NOCONV);
  // each phase's share: how far its last node finished after the previous
  // phase's last node (the phases overlap; the shares add up to the wall time)
  double prev = 0.0;
  for (int ph = 0; ph < 5; ++ph) {
    const double m = std::max(prev, last[ph]);
    S.section_ms[ph] += m - prev;
    prev = m;
  }
}

static void forward_euler(Solver& S, Exec& ex, const TT Q[3], unsigned seed, TT out[3]) {
  if (S.p.eqn == TT_LINEAR)
    forward_euler_linear(S, ex, Q, seed, out);
  else
    forward_euler_graph(S, ex, Q, seed, out);
}

// kick-index seed of a stage: depends on the stage and call site only, so a
// solver restarted from a checkpoint draws the same kicks
static unsigned stage_seed(const Solver& S, int stage) { return S.p.seed + 1000u * (unsigned)stage; }

// Truncation tolerances of a step (Sec. 4.4), from the step's input state:
// under TT_EPS_ADAPTIVE eps_u = min(1e-3, C V^(1/2) dx^(p-1/2) / ||u||_F) per
// field (Eq. modified-eps-tt-formula) and eps_TT = C V^(1/2) dx^(p-1/2) /
// max_q ||q||_F for the other rounds (Eq. eps-tt-formula); under
// TT_EPS_FIXED the fixed tol everywhere.
static void step_tolerances(Solver& S, Exec& ex) {
  if (S.p.eps_rule != TT_EPS_ADAPTIVE) {
    for (int c = 0; c < 3; ++c) S.tol_u[c] = S.p.tol;
    return;
  }
  Scope sc(*ex.ar);
  double* d = ex.ar->get<double>(8);
  for (int c = 0; c < 3; ++c) tt_sum_norm(ex, S.Qn[c], d + 2 * c);
  double v[6];
  fetch_doubles(ex, d, 6, v);
  const int order = S.p.recon == TT_UP3 ? 3 : 5;
  const double num = S.p.c_eps * std::sqrt(S.p.lx * S.p.ly) * std::pow(S.p.lx / S.p.nx, order - 0.5);
  double mx = 0.0;
  for (int c = 0; c < 3; ++c) {
    const double nrm = v[2 * c + 1];
    mx = std::max(mx, nrm);
    S.tol_u[c] = nrm > 0.0 ? std::min(1e-3, num / nrm) : 1e-3;
  }
  S.p.tol = mx > 0.0 ? num / mx : 1e-3;
}

static void run_stage(Solver& S, Exec& ex, int stage) {
  TT_REQUIRE(stage == S.next_stage, TT_ERR_ARG);
  TT_REQUIRE(S.p.bc_x != TT_BC_EXACT || S.boundary_set || ex.dry, TT_ERR_ARG);
  if (stage == 0) {
    step_tolerances(S, ex);
    // the lambda guesses and sketch widths carried between stages are
    // per-step state: a solver restarted from a checkpoint of Q (taken
    // between steps) repeats the next step bit for bit
    S.lam_prev_ok[0] = S.lam_prev_ok[1] = false;
    for (int d = 0; d < 2; ++d)
      for (int c = 0; c < 3; ++c) S.rf_hint[d][c] = 0;
  }
  Scope sc(*ex.ar);
  const tt_fv_params& p = S.p;
  TT f[3];
  for (int c = 0; c < 3; ++c) f[c] = alloc_tt(*ex.ar, p.nx, p.ny, p.rank_cap);
  // the stages of Eq. tt-ssprk3 evaluate L at t^n, t^n + dt and t^n + dt/2
  S.stage_time = S.time + (stage == 0 ? 0.0 : stage == 1 ? p.dt : 0.5 * p.dt);
  forward_euler(S, ex, S.Qs, stage_seed(S, stage), f);
  if (stage == 0) {
    for (int c = 0; c < 3; ++c) copy_tt(ex, f[c], S.Qs[c]);
  } else if (stage == 1) {
    SectionTimer st5(S.section_ms[5]);
    parallel_tasks(ex, 3, [&](Exec& cx, int c) {
      round_sum(cx, {Term{0.75, S.Qn[c]}, Term{0.25, f[c]}}, S.tol_u[c], p.rank_cap, S.Qs[c]);
    });
  } else {
    SectionTimer st5(S.section_ms[5]);
    parallel_tasks(ex, 3, [&](Exec& cx, int c) {
      round_sum(cx, {Term{1.0 / 3.0, S.Qn[c]}, Term{2.0 / 3.0, f[c]}}, S.tol_u[c], p.rank_cap, S.Qn[c]);
    });
    for (int c = 0; c < 3; ++c) copy_tt(ex, S.Qn[c], S.Qs[c]);
    S.step_count++;
    if (!ex.dry) S.time += p.dt;
  }
  S.next_stage = (stage + 1) % 3;
}

// ---------------------------------------------------------------- C ABI glue
static tt_status guard_status(Exec& ex) {
  if (ex.dry || ex.dev_status == nullptr) return TT_OK;
  unsigned st = 0;
  TT_CUDA(cudaMemcpyAsync(&st, ex.dev_status, sizeof(unsigned), cudaMemcpyDeviceToHost, ex.s));
  TT_CUDA(cudaStreamSynchronize(ex.s));
  prof_flush(ex);
  if (st & DEV_TC_TIMEOUT) return TT_ERR_TIMEOUT;
  if (st & DEV_NONFINITE) return TT_ERR_NONFINITE;
  if (st & DEV_JACOBI_NOCONV) return TT_ERR_NOCONV;
  return TT_OK;
}

static bool valid_params(const tt_fv_params* p) {
  if (!p) return false;
  if (p->eqn != TT_LINEAR && p->eqn != TT_NONLINEAR) return false;
  if (p->recon < TT_UP3 || p->recon > TT_WENO5) return false;
  if (p->nx < 8 || p->ny < 8 || p->rank_cap < 1 || p->rank_cap > 100) return false;
  if (!(p->tol >= 0.0) || !(p->dt > 0.0) || !(p->lx > 0.0) || !(p->ly > 0.0) || !(p->g > 0.0)) return false;
  if (p->precision < TT_FP64 || p->precision > TT_FP32) return false;
  if (p->pivots != TT_PIVOT_MAXVOL && p->pivots != TT_PIVOT_LEARNED) return false;
  if (p->eqn == TT_LINEAR && !(p->H > 0.0)) return false;
  if (p->eps_rule != TT_EPS_FIXED && p->eps_rule != TT_EPS_ADAPTIVE) return false;
  if (p->eps_rule == TT_EPS_ADAPTIVE && !(p->c_eps > 0.0)) return false;
  if (p->flux != TT_FLUX_PRODUCTS && p->flux != TT_FLUX_CROSS) return false;
  if (p->forcing_waves < 0 || p->forcing_waves > TT_MAX_WAVES) return false;
  if (p->bc_x != TT_BC_PERIODIC && p->bc_x != TT_BC_EXACT) return false;
  if (p->bc_x == TT_BC_EXACT &&
      (p->eqn != TT_LINEAR || p->recon == TT_WENO5 || p->boundary_waves < 1 || p->boundary_waves > TT_MAX_WAVES))
    return false;
  return true;
}

static bool valid_tt(const tt2* x) {
  return x && x->n1 >= 1 && x->n2 >= 1 && x->rank >= 1 && x->cap >= x->rank && x->a && x->b;
}

static TT to_tt(const tt2& x) {
  TT t;
  t.n1 = x.n1;
  t.n2 = x.n2;
  t.r = x.rank;
  t.cap = x.cap;
  t.a = x.a;
  t.b = x.b;
  return t;
}

// Sets up an Exec over caller workspace: first 256 bytes = device status.
static void setup_exec(Exec& ex, Arena& ar, void* ws, size_t ws_bytes, cudaStream_t s, int* hi, double* hd,
                       bool dry) {
  ar.base = static_cast<char*>(ws);
  ar.cap = ws_bytes;
  ar.off = 0;
  ar.dry = dry;
  ex.ar = &ar;
  ex.s = s;
  ex.dry = dry;
  ex.h_pinned = hi;
  ex.h_pinned_d = hd;
  ex.dev_status = ar.get<unsigned>(64);
  if (!dry) TT_CUDA(cudaMemsetAsync(ex.dev_status, 0, sizeof(unsigned), s));
}

// ---------------------------------------------------------------- call wrappers
template <typename F>
static size_t dry_bytes(F&& body) {
  Arena ar;
  Exec ex;
  int hi[16];
  double hd[16];
  setup_exec(ex, ar, nullptr, 0, nullptr, hi, hd, true);
  try {
    body(ex);
  } catch (const Error&) {
    return 0;
  }
  return ar.peak + ar.peak / 4 + (4u << 20);
}

template <typename F>
static tt_status run_call(void* ws, size_t ws_bytes, void* stream, F&& body) {
  if (!ws) return TT_ERR_ARG;
  Arena ar;
  Exec ex;
  int hi[16];
  double hd[16];
  try {
    setup_exec(ex, ar, ws, ws_bytes, static_cast<cudaStream_t>(stream), hi, hd, false);
    tt_status r = body(ex);
    if (r != TT_OK) return r;
    return guard_status(ex);
  } catch (const Error& e) {
    return e.code;
  }
}

}  // namespace ttfv

using namespace ttfv;

struct tt_fv_ctx {
  Solver S;
};

namespace ttfv {
// Batched form: whether an instance runs its independent stage tasks on its
// own pool of streams (off: in order on the instance stream).
void solver_task_pool(tt_fv_ctx* ctx, bool on) { ctx->S.ex.pool = on ? &ctx->S.pool : nullptr; }
}  // namespace ttfv

extern "C" {

const char* tt_fv_version(void) { return "tt_fv 0.2 (sm_103a, FP64 path + FP32/TF32/BF16 precision forms)"; }

// persistent state beside Q: the previous stage's lambda of each direction
static void alloc_lambda_prev(Solver& S) {
  if (S.p.eqn == TT_LINEAR) return;
  S.lam_prev[0] = alloc_tt(S.ar, S.p.nx, S.nq * S.p.ny, S.p.rank_cap);
  S.lam_prev[1] = alloc_tt(S.ar, S.nq * S.p.nx, S.p.ny, S.p.rank_cap);
}

// TSQR tile shapes a solver may be switched to after its workspace is sized
// (tt_fv_set_tile_shape): (leaf-row multiple, largest merge fan-in; 0 = the
// default, 4 from p = 32 up).  Entry 0 is the default of every Exec.
static const int kTiles[][2] = {{2, 0}, {1, 0}, {1, 2}, {2, 2}, {3, 0}, {4, 0}};
constexpr int kNumTiles = int(sizeof(kTiles) / sizeof(kTiles[0]));

static size_t solver_bytes_tiles(const tt_fv_params* p, int tile) {
  // dry run of one stage at the rank cap
  Solver S;
  S.p = *p;
  S.nq = nq_of(p->recon);
  Exec ex;
  int hi[16];
  double hd[16];
  setup_exec(ex, S.ar, nullptr, 0, nullptr, hi, hd, true);
  ex.qr_leaf_mult = kTiles[tile][0];
  ex.qr_fanin = kTiles[tile][1];
  ex.precision = p->precision;
  MlpNet dry_net;  // sizing pass: the proposal's scratch is counted, no weight is read
  if (p->pivots == TT_PIVOT_LEARNED) ex.pivot_net = &dry_net;
  try {
    for (int c = 0; c < 3; ++c) {
      S.Qn[c] = alloc_tt(S.ar, p->nx, p->ny, p->rank_cap);
      S.Qs[c] = alloc_tt(S.ar, p->nx, p->ny, p->rank_cap);
      S.Qn[c].r = S.Qs[c].r = p->rank_cap;
    }
    alloc_lambda_prev(S);
    for (int st = 0; st < 3; ++st) run_stage(S, ex, st);
  } catch (const Error&) {
    return 0;
  }
  return S.ar.peak;
}

// the largest footprint over the tile shapes, so that any of them fits
static size_t solver_bytes(const tt_fv_params* p) {
  size_t peak = 0;
  for (int t = 0; t < kNumTiles; ++t) {
    const size_t b = solver_bytes_tiles(p, t);
    if (b == 0) return 0;
    peak = std::max(peak, b);
  }
  return peak + peak / 2 + (64u << 20);
}

size_t tt_fv_workspace_size(const tt_fv_params* p) {
  if (!valid_params(p)) return 0;
  return solver_bytes(p);
}

int32_t tt_tile_shapes(int32_t* leaf_mult, int32_t* fanin, int32_t max) {
  for (int t = 0; t < kNumTiles && t < max; ++t) {
    if (leaf_mult) leaf_mult[t] = kTiles[t][0];
    if (fanin) fanin[t] = kTiles[t][1];
  }
  return kNumTiles;
}

tt_status tt_fv_set_tile_shape(tt_fv_ctx* ctx, int32_t shape) {
  if (!ctx || shape < 0 || shape >= kNumTiles) return TT_ERR_ARG;
  ctx->S.ex.qr_leaf_mult = kTiles[shape][0];
  ctx->S.ex.qr_fanin = kTiles[shape][1];
  return TT_OK;
}

tt_status tt_fv_init(const tt_fv_params* p, const tt2 q0[3], void* ws, size_t ws_bytes, void* stream,
                     tt_fv_ctx** out) {
  if (!out || !valid_params(p) || !q0 || !ws) return TT_ERR_ARG;
  for (int c = 0; c < 3; ++c)
    if (!valid_tt(&q0[c]) || q0[c].n1 != p->nx || q0[c].n2 != p->ny || q0[c].rank > p->rank_cap)
      return TT_ERR_ARG;
  tt_fv_ctx* ctx = new (std::nothrow) tt_fv_ctx();
  if (!ctx) return TT_ERR_OOM;
  Solver& S = ctx->S;
  S.p = *p;
  for (int c = 0; c < 3; ++c) S.tol_u[c] = p->tol;
  S.s = static_cast<cudaStream_t>(stream);
  S.nq = nq_of(p->recon);
  try {
    setup_exec(S.ex, S.ar, ws, ws_bytes, S.s, S.h_int, S.h_dbl, false);
    if (char* ps = S.pool.slot(0)) {
      S.ex.h_pinned = reinterpret_cast<int*>(ps);
      S.ex.h_pinned_d = reinterpret_cast<double*>(ps + 64);
    }
    S.ex.prof = &S.prof;
    S.ex.pool = &S.pool;
    S.ex.precision = p->precision;
    S.ex.svd_cluster = false;  // a stage runs many roundings at once
    for (int c = 0; c < 3; ++c) {
      S.Qn[c] = alloc_tt(S.ar, p->nx, p->ny, p->rank_cap);
      S.Qs[c] = alloc_tt(S.ar, p->nx, p->ny, p->rank_cap);
      copy_tt(S.ex, to_tt(q0[c]), S.Qn[c]);
      copy_tt(S.ex, to_tt(q0[c]), S.Qs[c]);
    }
    alloc_lambda_prev(S);
    S.ar.peak = S.ar.off;
  } catch (const Error& e) {
    delete ctx;
    return e.code;
  }
  *out = ctx;
  return TT_OK;
}

tt_status tt_fv_stage(tt_fv_ctx* ctx, int32_t stage) {
  if (!ctx || stage < 0 || stage > 2) return TT_ERR_ARG;
  try {
    run_stage(ctx->S, ctx->S.ex, stage);
    return guard_status(ctx->S.ex);
  } catch (const Error& e) {
    return e.code;
  }
}

tt_status tt_fv_step(tt_fv_ctx* ctx, int32_t nsteps) {
  if (!ctx || nsteps < 0 || ctx->S.next_stage != 0) return TT_ERR_ARG;
  for (int n = 0; n < nsteps; ++n)
    for (int st = 0; st < 3; ++st) {
      tt_status r = tt_fv_stage(ctx, st);
      if (r != TT_OK) return r;
    }
  return TT_OK;
}

tt_status tt_fv_get(tt_fv_ctx* ctx, tt2 q_out[3]) {
  if (!ctx || !q_out) return TT_ERR_ARG;
  Solver& S = ctx->S;
  try {
    for (int c = 0; c < 3; ++c) {
      const TT& src = S.Qs[c];
      if (!q_out[c].a || !q_out[c].b || q_out[c].n1 != src.n1 || q_out[c].n2 != src.n2 || q_out[c].cap < src.r)
        return TT_ERR_ARG;
      TT dst = to_tt(q_out[c]);
      dst.r = 0;
      copy_tt(S.ex, src, dst);
      q_out[c].rank = src.r;
    }
    TT_CUDA(cudaStreamSynchronize(S.s));
  } catch (const Error& e) {
    return e.code;
  }
  return TT_OK;
}

tt_status tt_fv_set(tt_fv_ctx* ctx, const tt2 q[3]) {
  if (!ctx || !q) return TT_ERR_ARG;
  Solver& S = ctx->S;
  for (int c = 0; c < 3; ++c)
    if (!valid_tt(&q[c]) || q[c].n1 != S.p.nx || q[c].n2 != S.p.ny || q[c].rank > S.p.rank_cap) return TT_ERR_ARG;
  try {
    for (int c = 0; c < 3; ++c) {
      copy_tt(S.ex, to_tt(q[c]), S.Qn[c]);
      copy_tt(S.ex, to_tt(q[c]), S.Qs[c]);
    }
    S.next_stage = 0;
  } catch (const Error& e) {
    return e.code;
  }
  return TT_OK;
}

tt_status tt_fv_set_forcing(tt_fv_ctx* ctx, const tt_wave* waves, int32_t nwaves, double t0) {
  if (!ctx || nwaves < 0 || (nwaves > 0 && !waves) || !std::isfinite(t0)) return TT_ERR_ARG;
  Solver& S = ctx->S;
  int per[3] = {0, 0, 0};
  for (int i = 0; i < nwaves; ++i) {
    const tt_wave& w = waves[i];
    if (w.field < 0 || w.field > 2 || !std::isfinite(w.amp) || !std::isfinite(w.kx) || !std::isfinite(w.ky) ||
        !std::isfinite(w.omega) || !std::isfinite(w.phase) || !std::isfinite(w.decay))
      return TT_ERR_ARG;
    if (++per[w.field] > S.p.forcing_waves) return TT_ERR_ARG;
  }
  S.waves.assign(waves, waves + nwaves);
  S.time = t0;
  return TT_OK;
}

tt_status tt_fv_set_boundary(tt_fv_ctx* ctx, const tt_wave* waves, int32_t nwaves, double t0) {
  if (!ctx || nwaves < 0 || (nwaves > 0 && !waves) || !std::isfinite(t0)) return TT_ERR_ARG;
  Solver& S = ctx->S;
  if (S.p.bc_x != TT_BC_EXACT) return TT_ERR_ARG;
  int per[3] = {0, 0, 0};
  for (int i = 0; i < nwaves; ++i) {
    const tt_wave& w = waves[i];
    if (w.field < 0 || w.field > 2 || !std::isfinite(w.amp) || !std::isfinite(w.kx) || !std::isfinite(w.ky) ||
        !std::isfinite(w.omega) || !std::isfinite(w.phase) || !std::isfinite(w.decay))
      return TT_ERR_ARG;
    if (++per[w.field] > S.p.boundary_waves) return TT_ERR_ARG;
  }
  S.bwaves.assign(waves, waves + nwaves);
  S.boundary_set = true;
  S.time = t0;
  return TT_OK;
}

tt_status tt_fv_stats_get(tt_fv_ctx* ctx, tt_fv_stats* o) {
  if (!ctx || !o) return TT_ERR_ARG;
  Solver& S = ctx->S;
  Exec& ex = S.ex;
  std::memset(o, 0, sizeof(*o));
  for (int c = 0; c < 3; ++c) o->rank[c] = S.Qs[c].r;
  o->rounds = ex.rounds;
  o->syncs = ex.syncs;
  o->jacobi_sweeps = ex.jacobi_sweeps;
  o->cross_calls = ex.cross_calls;
  o->cross_sweeps = ex.cross_sweeps;
  o->taylor_iters = ex.taylor_iters;
  o->cap_hits = ex.cap_hits;
  o->qb_attempts = ex.qb_attempts;
  o->qb_uncertified = ex.qb_uncertified;
  o->flops = ex.flops;
  o->bytes = ex.bytes;
  o->svd_calls = ex.svd_calls;
  o->svd_p_sum = ex.svd_p;
  o->svd_pd_sum = ex.svd_pd;
  o->svd_sweeps_sum = ex.svd_sweeps;
  o->learned_calls = ex.learned_calls;
  o->learned_accepted = ex.learned_accepted;
  for (int i = 0; i < 6; ++i) o->section_ms[i] = S.section_ms[i];
  for (int c = 0; c < 3; ++c) o->eps_u[c] = S.tol_u[c];
  o->eps_tt = S.p.tol;
  unsigned st = 0;
  if (cudaMemcpyAsync(&st, ex.dev_status, sizeof(unsigned), cudaMemcpyDeviceToHost, S.s) != cudaSuccess ||
      cudaStreamSynchronize(S.s) != cudaSuccess)
    return TT_ERR_CUDA;
  o->device_status = st;
  return TT_OK;
}

tt_status tt_fv_set_pivot_net(tt_fv_ctx* ctx, const tt_mlp* net) {
  if (!ctx) return TT_ERR_ARG;
  Solver& S = ctx->S;
  if (!net) {
    S.ex.pivot_net = nullptr;
    return TT_OK;
  }
  if (S.p.pivots != TT_PIVOT_LEARNED || !net->W1 || !net->b1 || !net->W2 || !net->b2 || !net->w3 || !net->b3)
    return TT_ERR_ARG;
  S.net.W1 = net->W1;
  S.net.b1 = net->b1;
  S.net.W2 = net->W2;
  S.net.b2 = net->b2;
  S.net.w3 = net->w3;
  S.net.b3 = net->b3;
  S.ex.pivot_net = &S.net;
  return TT_OK;
}

tt_status tt_fv_record_pivots(tt_fv_ctx* ctx, int32_t enable) {
  if (!ctx) return TT_ERR_ARG;
  Solver& S = ctx->S;
  delete S.rec;
  S.rec = enable ? new (std::nothrow) PivotRecorder() : nullptr;
  if (enable && !S.rec) return TT_ERR_OOM;
  S.ex.pivot_rec = S.rec;
  return TT_OK;
}

int64_t tt_fv_pivot_rows(tt_fv_ctx* ctx) {
  if (!ctx || !ctx->S.rec) return 0;
  std::lock_guard<std::mutex> lk(ctx->S.rec->mu);
  return (int64_t)ctx->S.rec->y.size();
}

tt_status tt_fv_pivot_take(tt_fv_ctx* ctx, float* X, float* y, int64_t rows) {
  if (!ctx || !ctx->S.rec || !X || !y) return TT_ERR_ARG;
  PivotRecorder& R = *ctx->S.rec;
  std::lock_guard<std::mutex> lk(R.mu);
  if (rows != (int64_t)R.y.size()) return TT_ERR_ARG;
  std::memcpy(X, R.X.data(), sizeof(float) * R.X.size());
  std::memcpy(y, R.y.data(), sizeof(float) * R.y.size());
  R.X.clear();
  R.y.clear();
  return TT_OK;
}

void tt_fv_destroy(tt_fv_ctx* ctx) { delete ctx; }

tt_status tt_fv_profile(tt_fv_ctx* ctx, int32_t enable) {
  if (!ctx) return TT_ERR_ARG;
  try {
    TT_CUDA(cudaStreamSynchronize(ctx->S.s));
    prof_flush(ctx->S.ex);
  } catch (const Error& e) {
    return e.code;
  }
  ctx->S.prof.on = enable != 0;
  return TT_OK;
}

tt_status tt_fv_kernel_profile(tt_fv_ctx* ctx, tt_kernel_prof out[TT_K_NCLASS], int32_t reset) {
  if (!ctx || !out) return TT_ERR_ARG;
  Prof& pf = ctx->S.prof;
  try {
    TT_CUDA(cudaStreamSynchronize(ctx->S.s));
    prof_flush(ctx->S.ex);
  } catch (const Error& e) {
    return e.code;
  }
  for (int c = 0; c < TT_K_NCLASS; ++c) {
    out[c].ms = pf.ms[c];
    out[c].flops = pf.flops[c];
    out[c].bytes = pf.bytes[c];
    out[c].launches = pf.n[c];
    if (reset) {
      pf.ms[c] = pf.flops[c] = pf.bytes[c] = 0.0;
      pf.n[c] = 0;
    }
  }
  return TT_OK;
}

uint64_t tt_launch_count(void) { return g_launches.load(); }

// ---------------------------------------------------------------- primitives
static TT fake_tt(Arena& ar, int n1, int n2, int r) {
  TT t = alloc_tt(ar, n1, n2, r);
  t.r = r;
  return t;
}

size_t tt_round_workspace_size(int32_t n1, int32_t n2, int32_t rank_in, int32_t rank_cap) {
  if (n1 < 1 || n2 < 1 || rank_in < 1 || rank_cap < 1) return 0;
  return dry_bytes([&](Exec& ex) {
    TT x = fake_tt(*ex.ar, n1, n2, rank_in);
    TT y = fake_tt(*ex.ar, n1, n2, rank_cap);
    round_tt(ex, x, 0.0, rank_cap, y);
  });
}

tt_status tt_round(const tt2* x, double tol, int32_t rank_cap, tt2* y, double* err_out, void* ws, size_t ws_bytes,
                   void* stream) {
  if (!valid_tt(x) || !y || !y->a || !y->b || y->n1 != x->n1 || y->n2 != x->n2 || rank_cap < 1 ||
      y->cap < std::min(rank_cap, std::min(x->n1, x->n2)) || !(tol >= 0.0))
    return TT_ERR_ARG;
  return run_call(ws, ws_bytes, stream, [&](Exec& ex) {
    TT X = to_tt(*x), Y = to_tt(*y);
    RoundInfo ri = round_tt(ex, X, tol, rank_cap, Y);
    y->rank = Y.r;
    if (err_out) *err_out = ri.err;
    return TT_OK;
  });
}

size_t tt_round_hadamard_workspace_size(int32_t n1, int32_t n2, int32_t rank_x, int32_t rank_z, int32_t rank_cap) {
  if (n1 < 1 || n2 < 1 || rank_x < 1 || rank_z < 1 || rank_cap < 1) return 0;
  return dry_bytes([&](Exec& ex) {
    TT x = fake_tt(*ex.ar, n1, n2, rank_x), z = fake_tt(*ex.ar, n1, n2, rank_z);
    TT y = fake_tt(*ex.ar, n1, n2, rank_cap);
    round_hadamard(ex, x, z, 0.0, rank_cap, y);
  });
}

tt_status tt_round_hadamard(const tt2* x, const tt2* z, double tol, int32_t rank_cap, tt2* y, void* ws,
                            size_t ws_bytes, void* stream) {
  if (!valid_tt(x) || !valid_tt(z) || !y || !y->a || !y->b || x->n1 != z->n1 || x->n2 != z->n2 ||
      y->n1 != x->n1 || y->n2 != x->n2 || rank_cap < 1 || y->cap < std::min(rank_cap, std::min(x->n1, x->n2)) ||
      !(tol >= 0.0))
    return TT_ERR_ARG;
  return run_call(ws, ws_bytes, stream, [&](Exec& ex) {
    TT X = to_tt(*x), Z = to_tt(*z), Y = to_tt(*y);
    round_hadamard(ex, X, Z, tol, rank_cap, Y);
    y->rank = Y.r;
    return TT_OK;
  });
}

// ---------------------------------------------------------------- dense contraction
}  // extern "C"
namespace ttfv {
__global__ void k_pack_cols(const double* __restrict__ X, long ld, int m, int n, float* __restrict__ Y) {
  const long total = (long)m * n;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x)
    Y[t] = (float)X[(t % m) + (t / m) * ld];
}
__global__ void k_axpby_f32(int m, int n, double alpha, const float* __restrict__ P, double beta,
                            double* __restrict__ C, long ldc) {
  const long total = (long)m * n;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    double* c = C + (t % m) + (size_t)(t / m) * ldc;
    *c = (beta == 0.0) ? alpha * (double)P[t] : fma(alpha, (double)P[t], beta * *c);
  }
}
static void contract(Exec& ex, int precision, int split, int m, int n, int k, double alpha, const double* A, long lda,
                     const double* B, long ldb, double beta, double* C, long ldc) {
  if (precision == TT_FP64) {
    gemm<double>(ex, m, n, k, alpha, A, 1, lda, B, 1, ldb, beta, C, ldc);
    return;
  }
  Scope sc(*ex.ar);
  float* P = ex.ar->get<float>((size_t)m * n);
  if (precision == TT_FP32) {
    float* A32 = ex.ar->get<float>((size_t)m * k);
    float* B32 = ex.ar->get<float>((size_t)k * n);
    if (!ex.dry) {
      const int gA = std::max(1, std::min(ceil_div((long)m * k, 256), 1184));
      const int gB = std::max(1, std::min(ceil_div((long)k * n, 256), 1184));
      TT_KERNEL(ex, K_OTHER, 0, 12.0 * m * k, k_pack_cols<<<gA, 256, 0, ex.s>>>(A, lda, m, k, A32));
      TT_KERNEL(ex, K_OTHER, 0, 12.0 * k * n, k_pack_cols<<<gB, 256, 0, ex.s>>>(B, ldb, k, n, B32));
    }
    gemm<float>(ex, m, n, k, 1.0f, A32, 1, m, B32, 1, k, 0.0f, P, m);
  } else {
    tc_gemm<double>(ex, precision, split != 0, m, n, k, 1.0f, A, 1, lda, B, 1, ldb, 0.0f, P, m);
  }
  if (ex.dry) return;
  const long total = (long)m * n;
  TT_KERNEL(ex, K_OTHER, 2.0 * total, 16.0 * total + 4.0 * total,
            k_axpby_f32<<<std::max(1, std::min(ceil_div(total, 256), 1184)), 256, 0, ex.s>>>(m, n, alpha, P, beta,
                                                                                               C, ldc));
}
}  // namespace ttfv
extern "C" {

size_t tt_contract_workspace_size(int32_t precision, int32_t split, int32_t m, int32_t n, int32_t k) {
  if (precision < TT_FP64 || precision > TT_FP32 || m < 1 || n < 1 || k < 1) return 0;
  return dry_bytes([&](Exec& ex) { contract(ex, precision, split, m, n, k, 1.0, nullptr, m, nullptr, k, 0.0,
                                            nullptr, m); });
}

tt_status tt_contract(int32_t precision, int32_t split, int32_t m, int32_t n, int32_t k, double alpha,
                      const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                      void* ws, size_t ws_bytes, void* stream) {
  if (precision < TT_FP64 || precision > TT_FP32 || m < 1 || n < 1 || k < 1 || !A || !B || !C || lda < m ||
      ldb < k || ldc < m)
    return TT_ERR_ARG;
  return run_call(ws, ws_bytes, stream, [&](Exec& ex) {
    contract(ex, precision, split, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    return TT_OK;
  });
}

// ---------------------------------------------------------------- learned-pivot network
static bool valid_net(const tt_mlp* n) { return n && n->W1 && n->b1 && n->W2 && n->b2 && n->w3 && n->b3; }
static MlpNet to_net(const tt_mlp* n) {
  MlpNet m;
  m.W1 = n->W1;
  m.b1 = n->b1;
  m.W2 = n->W2;
  m.b2 = n->b2;
  m.w3 = n->w3;
  m.b3 = n->b3;
  return m;
}

size_t tt_mlp_workspace_size(int32_t rows, int32_t rank) {
  if (rows < 1 || rank < 1 || rank > 112) return 0;
  return dry_bytes([&](Exec& ex) {
    TT x0 = fake_tt(*ex.ar, rows, rows, rank);
    float* X = ex.ar->get<float>((size_t)rows * kMlpFeatures);
    float* y = ex.ar->get<float>((size_t)rows);
    mlp_features(ex, x0, nullptr, 0, X);
    MlpNet n, g;
    mlp_grad(ex, n, X, y, rows, g, nullptr);
    mlp_topk(ex, y, rows, std::min(rows, 112), nullptr);
  });
}

tt_status tt_mlp_features(const tt2* x0, const int32_t* prev, int32_t nprev, float* X, void* ws, size_t ws_bytes,
                          void* stream) {
  if (!valid_tt(x0) || x0->rank > 112 || !X || nprev < 0 || (nprev > 0 && !prev)) return TT_ERR_ARG;
  return run_call(ws, ws_bytes, stream, [&](Exec& ex) {
    mlp_features(ex, to_tt(*x0), prev, nprev, X);
    return TT_OK;
  });
}

tt_status tt_mlp_forward(const tt_mlp* net, const float* X, int32_t m, float* s, void* ws, size_t ws_bytes,
                         void* stream) {
  if (!valid_net(net) || !X || !s || m < 1) return TT_ERR_ARG;
  return run_call(ws, ws_bytes, stream, [&](Exec& ex) {
    mlp_forward(ex, to_net(net), X, m, s);
    return TT_OK;
  });
}

tt_status tt_mlp_grad(const tt_mlp* net, const float* X, const float* y, int32_t m, const tt_mlp* grad, double* loss,
                      void* ws, size_t ws_bytes, void* stream) {
  if (!valid_net(net) || !valid_net(grad) || !X || !y || m < 1) return TT_ERR_ARG;
  return run_call(ws, ws_bytes, stream, [&](Exec& ex) {
    mlp_grad(ex, to_net(net), X, y, m, to_net(grad), loss);
    return TT_OK;
  });
}

tt_status tt_mlp_adam(const tt_mlp* net, const tt_mlp* grad, const tt_mlp* m1, const tt_mlp* m2, int32_t t, float lr,
                      void* stream) {
  if (!valid_net(net) || !valid_net(grad) || !valid_net(m1) || !valid_net(m2) || t < 1 || !(lr > 0.0f))
    return TT_ERR_ARG;
  Arena ar;
  Exec ex;
  int hi[16];
  double hd[16];
  try {
    ar.dry = false;
    ex.ar = &ar;
    ex.s = static_cast<cudaStream_t>(stream);
    ex.h_pinned = hi;
    ex.h_pinned_d = hd;
    mlp_adam(ex, to_net(net), to_net(grad), to_net(m1), to_net(m2), t, lr);
  } catch (const Error& e) {
    return e.code;
  }
  return TT_OK;
}

tt_status tt_mlp_topk(const float* s, int32_t m, int32_t k, int32_t* idx, void* ws, size_t ws_bytes, void* stream) {
  if (!s || !idx || m < 1 || k < 1 || k > 128 || k > m) return TT_ERR_ARG;
  return run_call(ws, ws_bytes, stream, [&](Exec& ex) {
    mlp_topk(ex, s, m, k, idx);
    return TT_OK;
  });
}

size_t tt_cross_workspace_size(int32_t n1, int32_t n2, int32_t rank_in, int32_t rank_cap, int32_t kick) {
  if (n1 < 1 || n2 < 1 || rank_in < 1 || rank_cap < 1 || kick < 0) return 0;
  return dry_bytes([&](Exec& ex) {
    TT x0 = fake_tt(*ex.ar, n1, n2, rank_in);
    TT y = fake_tt(*ex.ar, n1, n2, rank_cap);
    CrossFn f;
    f.fn = TT_FN_ENTRY;
    f.in = &x0;
    f.nin = 1;
    cross(ex, f, n1, n2, x0, 0.0, rank_cap, kick, 2, 0, y);
  });
}

tt_status tt_cross(int32_t fn, const tt2* inputs, int32_t ninputs, const tt2* x0, const double* fparams, double tol,
                   int32_t rank_cap, int32_t kick, int32_t max_sweeps, uint32_t seed, tt2* y, int32_t* sweeps_out,
                   void* ws, size_t ws_bytes, void* stream) {
  if (fn < TT_FN_ENTRY || fn > TT_FN_LLF_FLUX || !inputs || ninputs < 1 || ninputs > 6 || !valid_tt(x0) || !y ||
      !y->a || !y->b || rank_cap < 1 || kick < 0 || max_sweeps < 1 || x0->n2 != y->n2 || !(tol >= 0.0) ||
      y->cap < rank_cap)
    return TT_ERR_ARG;
  const int need = fn == TT_FN_LLF_LAMBDA ? 4 : fn == TT_FN_LLF_FLUX ? 6 : 1;
  if (ninputs != need) return TT_ERR_ARG;
  for (int q = 0; q < ninputs; ++q) {
    if (!valid_tt(&inputs[q])) return TT_ERR_ARG;
    // every evaluated entry must index inside the inputs
    int e1 = y->n1, e2 = y->n2;
    if (fn == TT_FN_WENO_S2) {
      if (!fparams || fparams[2] != 3.0) return TT_ERR_ARG;
      if (fparams[1] == 1.0)
        e2 = 3 * inputs[q].n2;
      else if (fparams[1] == 0.0)
        e1 = 3 * inputs[q].n1;
      else
        return TT_ERR_ARG;
      if (y->n1 != e1 || y->n2 != e2) return TT_ERR_ARG;
    } else if (fn == TT_FN_LLF_FLUX) {
      if (3 * inputs[q].n1 != e1 || inputs[q].n2 != e2) return TT_ERR_ARG;
    } else if (inputs[q].n1 != e1 || inputs[q].n2 != e2) {
      return TT_ERR_ARG;
    }
  }
  if (fn == TT_FN_LLF_FLUX && (!fparams || (fparams[1] != 0.0 && fparams[1] != 1.0))) return TT_ERR_ARG;
  if (fn == TT_FN_WENO_S1 && (fparams[2] != 0.0 && fparams[2] != 1.0)) return TT_ERR_ARG;
  if ((fn == TT_FN_WENO_S1 || fn == TT_FN_WENO_S2 || fn == TT_FN_ENTRY) && !fparams && fn != TT_FN_ENTRY)
    return TT_ERR_ARG;
  if (fn == TT_FN_LLF_LAMBDA && !fparams) return TT_ERR_ARG;
  return run_call(ws, ws_bytes, stream, [&](Exec& ex) {
    TT ins[6];
    for (int q = 0; q < ninputs; ++q) ins[q] = to_tt(inputs[q]);
    CrossFn f;
    f.fn = fn;
    f.in = ins;
    f.nin = ninputs;
    if (fparams)
      for (int q = 0; q < 3; ++q) f.prm[q] = fparams[q];
    if (fn == TT_FN_LLF_LAMBDA) f.prm[0] = fparams[0];
    if (fn == TT_FN_LLF_FLUX) {
      f.prm[0] = fparams[0];
      f.prm[1] = fparams[1];
    }
    TT X0 = to_tt(*x0), Y = to_tt(*y);
    const int sw = cross(ex, f, y->n1, y->n2, X0, tol, rank_cap, kick, max_sweeps, seed, Y);
    y->rank = Y.r;
    if (sweeps_out) *sweeps_out = sw;
    return TT_OK;
  });
}

size_t tt_maxvol_workspace_size(int32_t n, int32_t r) {
  if (r < 1 || r > 128 || n < r) return 0;
  return dry_bytes([&](Exec& ex) { maxvol(ex, nullptr, n, r, 1e-2, 1, nullptr); });
}

tt_status tt_maxvol(const double* U, int32_t n, int32_t r, double delta, int32_t max_iter, int32_t* I, void* ws,
                    size_t ws_bytes, void* stream) {
  if (!U || !I || r < 1 || r > 128 || n < r || !(delta >= 0.0) || max_iter < 0) return TT_ERR_ARG;
  return run_call(ws, ws_bytes, stream, [&](Exec& ex) {
    maxvol(ex, U, n, r, delta, max_iter, I);
    return TT_OK;
  });
}

size_t tt_reciprocal_workspace_size(int32_t n1, int32_t n2, int32_t rank_in, int32_t rank_cap) {
  if (n1 < 1 || n2 < 1 || rank_in < 1 || rank_cap < 1) return 0;
  return dry_bytes([&](Exec& ex) {
    TT x = fake_tt(*ex.ar, n1, n2, rank_in);
    TT y = fake_tt(*ex.ar, n1, n2, rank_cap);
    reciprocal(ex, x, 1e-12, rank_cap, 2, y, nullptr);
  });
}

tt_status tt_reciprocal(const tt2* x, double tol, int32_t rank_cap, int32_t max_iter, tt2* y, int32_t* iters_out,
                        void* ws, size_t ws_bytes, void* stream) {
  if (!valid_tt(x) || !y || !y->a || !y->b || y->n1 != x->n1 || y->n2 != x->n2 || rank_cap < 1 ||
      y->cap < rank_cap || max_iter < 1 || !(tol > 0.0))
    return TT_ERR_ARG;
  return run_call(ws, ws_bytes, stream, [&](Exec& ex) {
    TT X = to_tt(*x), Y = to_tt(*y);
    bool nc = false;
    const int it = reciprocal(ex, X, tol, rank_cap, max_iter, Y, &nc);
    y->rank = Y.r;
    if (iters_out) *iters_out = it;
    return nc ? TT_ERR_NOCONV : TT_OK;
  });
}

tt_status tt_recon_linear(const tt2* x, int32_t direction, int32_t scheme, tt2* qm, tt2* qp, void* stream) {
  if (!valid_tt(x) || !qm || !qp || (direction != 0 && direction != 1) || (scheme != TT_UP3 && scheme != TT_UP5))
    return TT_ERR_ARG;
  const int nq = nq_of(scheme);
  const int f1 = direction == 0 ? x->n1 : nq * x->n1, f2 = direction == 0 ? nq * x->n2 : x->n2;
  for (tt2* q : {qm, qp})
    if (!q->a || !q->b || q->n1 != f1 || q->n2 != f2 || q->cap < x->rank) return TT_ERR_ARG;
  Arena ar;
  Exec ex;
  int hi[16];
  double hd[16];
  try {
    ar.dry = false;
    ex.ar = &ar;
    ex.s = static_cast<cudaStream_t>(stream);
    ex.h_pinned = hi;
    ex.h_pinned_d = hd;
    TT X = to_tt(*x), M = to_tt(*qm), P = to_tt(*qp);
    double* shared_keep = direction == 0 ? P.b : P.a;
    recon_linear(ex, X, direction, scheme, M, P);
    // the library shares the stacked core between qm and qp; the C ABI hands
    // the caller two independent copies
    if (direction == 0)
      scaled_copy(ex, shared_keep, M.b, (long)f2 * x->rank, 1.0);
    else
      scaled_copy(ex, shared_keep, M.a, (long)f1 * x->rank, 1.0);
    qm->rank = qp->rank = x->rank;
  } catch (const Error& e) {
    return e.code;
  }
  return TT_OK;
}

}  // extern "C"
