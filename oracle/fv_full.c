/* Oracle A in plain C: the full-tensor finite-volume discretisation of Sec. 2
 * (Danis et al., arXiv 2408.03483), for long runs and large grids where the
 * numpy form (fv_full.py) is too slow.
 *
 * TEST INFRASTRUCTURE ONLY: called from tests/ and from bench.py's oracle
 * legs through oracle/fv_c.py; it shares no code with the CUDA path.
 *
 * It computes what fv_full.py computes, step for step:
 *   Step 1 "de-cell" along the face normal (Sec. 2.3.1): the linear Upwind3 /
 *     Upwind5 stencils, or WENO5 with alpha_r = d_r / (beta_r + eps)^2;
 *     "+" side the mirror image of the "-" side;
 *   Step 2 to the Gauss points along the face (Sec. 2.3.2, Eq.
 *     fv-recon-step2): candidates sum_l c^m_{rl} v_{j-r+l}, linear weights or
 *     WENO5 weights gamma / (beta + eps)^2, the split of Eq.
 *     neg-coeff-treatment at the centre point of the 3-point rule;
 *   the LLF flux of Eq. LLF per Gauss point with lambda the larger of
 *     |u_n| + sqrt(g h) over the two states (sqrt(g H) for the linear SWE),
 *     the Gauss-Legendre face average, the difference (T - 1) F / dx of
 *     Eq. SWE-system-TT, and the source (0, f q2, -f q1);
 *   SSP-RK3 (Eq. tt-ssprk3 without rounding).
 * The coefficient tables come in from oracle/coeffs.py (fv_coeffs below), so
 * both forms of Oracle A read the same exact C^m, gamma and Gauss rule.
 *
 * Arrays are C-ordered nx x ny: U[i * ny + j], i the x cell, j the y cell;
 * periodic in both directions.  A face array F[i] holds the flux on the face
 * x_{i-1/2}, between cells i-1 and i.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int nq;             /* Gauss points per face: 2 (Upwind3) or 3 */
  int weno;           /* 1: WENO5 weights, 0: the linear weights */
  double lin1[2][5];  /* Step-1 linear stencils, side "-" (0) and "+" (1), offsets -2..2 */
  double C[3][3][3];  /* Step-2 C^m[r][l] */
  double gam[3][3];   /* Step-2 linear weights gamma_m^r (unused at the split point) */
  int split[3];       /* 1 at the Gauss point whose weights are split */
  double gp[3], gm[3], sp, sm; /* the split weights gamma^+, gamma^- and sigma^+, sigma^- */
  double w[3];        /* Gauss weights, summing to 1 */
} fv_coeffs;

typedef struct {
  int eqn;            /* 0 linear, 1 nonlinear */
  int nx, ny;
  double dx, dy, g, H, f;
} fv_grid;

static inline long idx(int i, int j, int ny) { return (long)i * ny + j; }

/* value of v shifted by s along axis at (i, j): v[i + s, j] or v[i, j + s] */
static inline double sh(const double* v, int i, int j, int s, int axis, int nx, int ny) {
  if (axis == 0) {
    int k = (i + s) % nx;
    if (k < 0) k += nx;
    return v[idx(k, j, ny)];
  }
  int k = (j + s) % ny;
  if (k < 0) k += ny;
  return v[idx(i, k, ny)];
}

static void betas(const double S[5], double b[3]) {
  const double vm2 = S[0], vm1 = S[1], v0 = S[2], vp1 = S[3], vp2 = S[4];
  double a, c;
  a = v0 - 2.0 * vp1 + vp2;
  c = 3.0 * v0 - 4.0 * vp1 + vp2;
  b[0] = 13.0 / 12.0 * a * a + 0.25 * c * c;
  a = vm1 - 2.0 * v0 + vp1;
  c = vm1 - vp1;
  b[1] = 13.0 / 12.0 * a * a + 0.25 * c * c;
  a = vm2 - 2.0 * vm1 + v0;
  c = vm2 - 4.0 * vm1 + 3.0 * v0;
  b[2] = 13.0 / 12.0 * a * a + 0.25 * c * c;
}

/* WENO5 "-" side value at x_{i+1/2} from v_{i-2..i+2} (Sec. 2.3.1) */
static double weno5_step1(const double S[5], double eps) {
  const double vm2 = S[0], vm1 = S[1], v0 = S[2], vp1 = S[3], vp2 = S[4];
  const double q0 = (2.0 * v0 + 5.0 * vp1 - vp2) / 6.0;
  const double q1 = (-vm1 + 5.0 * v0 + 2.0 * vp1) / 6.0;
  const double q2 = (2.0 * vm2 - 7.0 * vm1 + 11.0 * v0) / 6.0;
  double b[3];
  betas(S, b);
  const double a0 = 0.3 / ((b[0] + eps) * (b[0] + eps));
  const double a1 = 0.6 / ((b[1] + eps) * (b[1] + eps));
  const double a2 = 0.1 / ((b[2] + eps) * (b[2] + eps));
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

/* Step 1 along axis; side 0 "-" (value at the cell's upper face), 1 "+" */
static void step1(const double* v, double* out, const fv_grid* G, const fv_coeffs* co, int axis, int side,
                  double eps) {
  const int nx = G->nx, ny = G->ny;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < ny; ++j) {
      double S[5];
      for (int s = -2; s <= 2; ++s) S[s + 2] = sh(v, i, j, s, axis, nx, ny);
      double r;
      if (!co->weno) {
        r = 0.0;
        for (int s = 0; s < 5; ++s) r += co->lin1[side][s] * S[s];
      } else if (side == 0) {
        r = weno5_step1(S, eps);
      } else {
        const double M[5] = {S[4], S[3], S[2], S[1], S[0]};
        r = weno5_step1(M, eps);
      }
      out[idx(i, j, ny)] = r;
    }
}

/* Step 2 along axis to the nq Gauss points: out[m * n + cell] */
static void step2(const double* v, double* out, const fv_grid* G, const fv_coeffs* co, int axis, double eps) {
  const int nx = G->nx, ny = G->ny, nq = co->nq, k = nq - 1;
  const long n = (long)nx * ny;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < ny; ++j) {
      double S[5];
      for (int s = -2; s <= 2; ++s) S[s + 2] = sh(v, i, j, s, axis, nx, ny);
      double b[3] = {0.0, 0.0, 0.0};
      if (co->weno) betas(S, b);
      for (int m = 0; m < nq; ++m) {
        double cand[3];
        for (int r = 0; r <= k; ++r) {
          double c = 0.0;
          for (int l = 0; l <= k; ++l) c += co->C[m][r][l] * S[2 - r + l];
          cand[r] = c;
        }
        double val;
        if (!co->split[m]) {
          if (co->weno) {
            double a[3], as = 0.0, num = 0.0;
            for (int r = 0; r < 3; ++r) {
              a[r] = co->gam[m][r] / ((b[r] + eps) * (b[r] + eps));
              as += a[r];
              num += a[r] * cand[r];
            }
            val = num / as;
          } else {
            val = 0.0;
            for (int r = 0; r <= k; ++r) val += co->gam[m][r] * cand[r];
          }
        } else {
          double up, um;
          if (co->weno) {
            double ap = 0.0, am = 0.0, np_ = 0.0, nm = 0.0;
            for (int r = 0; r < 3; ++r) {
              const double d2 = (b[r] + eps) * (b[r] + eps);
              const double xp = co->gp[r] / d2, xm = co->gm[r] / d2;
              ap += xp;
              am += xm;
              np_ += xp * cand[r];
              nm += xm * cand[r];
            }
            up = np_ / ap;
            um = nm / am;
          } else {
            up = um = 0.0;
            for (int r = 0; r < 3; ++r) {
              up += co->gp[r] * cand[r];
              um += co->gm[r] * cand[r];
            }
          }
          val = co->sp * up - co->sm * um;
        }
        out[(long)m * n + idx(i, j, ny)] = val;
      }
    }
}

/* physical flux of Eq. linear-SWE / nonlinear-SWE in direction dir */
static inline void phys_flux(const fv_grid* G, int dir, const double q[3], double F[3]) {
  if (G->eqn == 0) {
    if (dir == 0) {
      F[0] = G->H * q[1];
      F[1] = G->g * q[0];
      F[2] = 0.0;
    } else {
      F[0] = G->H * q[2];
      F[1] = 0.0;
      F[2] = G->g * q[0];
    }
    return;
  }
  const double h = q[0], hu = q[1], hv = q[2];
  if (dir == 0) {
    F[0] = hu;
    F[1] = hu * hu / h + 0.5 * G->g * h * h;
    F[2] = hu * hv / h;
  } else {
    F[0] = hv;
    F[1] = hu * hv / h;
    F[2] = hv * hv / h + 0.5 * G->g * h * h;
  }
}

static inline double speed(const fv_grid* G, int dir, const double qm[3], const double qp[3]) {
  if (G->eqn == 0) return sqrt(G->g * G->H);
  const int k = dir == 0 ? 1 : 2;
  const double lm = fabs(qm[k] / qm[0]) + sqrt(G->g * qm[0]);
  const double lp = fabs(qp[k] / qp[0]) + sqrt(G->g * qp[0]);
  return lm > lp ? lm : lp;
}

/* L(Q) of Eq. SWE-system-cell-avg into L[3] (work: 2 * 3 * nq * n + 4 n doubles) */
static void rhs(const fv_grid* G, const fv_coeffs* co, double* const Q[3], double* L[3], double* work) {
  const int nx = G->nx, ny = G->ny, nq = co->nq;
  const long n = (long)nx * ny;
  double* right = work;             /* 3 x nq x n: Step 2 of the "-" side */
  double* left = right + 3 * nq * n; /* 3 x nq x n: Step 2 of the "+" side */
  double* s1 = left + 3 * nq * n;   /* n */
  double* Fq = s1 + n;              /* 3 x n */
  for (int c = 0; c < 3; ++c) memset(L[c], 0, sizeof(double) * n);
  for (int dir = 0; dir < 2; ++dir) {
    const int a1 = dir, a2 = 1 - dir;
    const double e1 = dir == 0 ? G->dx * G->dx : G->dy * G->dy;
    const double e2 = dir == 0 ? G->dy * G->dy : G->dx * G->dx;
    const double d = dir == 0 ? G->dx : G->dy;
    for (int c = 0; c < 3; ++c) {
      step1(Q[c], s1, G, co, a1, 0, e1);
      step2(s1, right + (long)c * nq * n, G, co, a2, e2);
      step1(Q[c], s1, G, co, a1, 1, e1);
      step2(s1, left + (long)c * nq * n, G, co, a2, e2);
    }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nx; ++i)
      for (int j = 0; j < ny; ++j) {
        /* the state left of the face is the previous cell's "-" value */
        const int ip = dir == 0 ? (i - 1 + nx) % nx : i;
        const int jp = dir == 0 ? j : (j - 1 + ny) % ny;
        double acc[3] = {0.0, 0.0, 0.0};
        for (int m = 0; m < nq; ++m) {
          double qm[3], qp[3], Fm[3], Fp[3];
          for (int c = 0; c < 3; ++c) {
            qm[c] = right[((long)c * nq + m) * n + idx(ip, jp, ny)];
            qp[c] = left[((long)c * nq + m) * n + idx(i, j, ny)];
          }
          phys_flux(G, dir, qm, Fm);
          phys_flux(G, dir, qp, Fp);
          const double lam = speed(G, dir, qm, qp);
          for (int c = 0; c < 3; ++c)
            acc[c] += co->w[m] * (0.5 * (Fm[c] + Fp[c]) - 0.5 * lam * (qp[c] - qm[c]));
        }
        for (int c = 0; c < 3; ++c) Fq[(long)c * n + idx(i, j, ny)] = acc[c];
      }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nx; ++i)
      for (int j = 0; j < ny; ++j) {
        const int in = dir == 0 ? (i + 1) % nx : i;
        const int jn = dir == 0 ? j : (j + 1) % ny;
        for (int c = 0; c < 3; ++c)
          L[c][idx(i, j, ny)] -= (Fq[(long)c * n + idx(in, jn, ny)] - Fq[(long)c * n + idx(i, j, ny)]) / d;
      }
  }
  /* the source (0, f q2, -f q1) is linear in Q: its cell average is S(Q) */
#pragma omp parallel for schedule(static)
  for (long t = 0; t < n; ++t) {
    L[1][t] += G->f * Q[2][t];
    L[2][t] -= G->f * Q[1][t];
  }
}

/* nsteps SSP-RK3 steps of size dt on Q (3 arrays of nx * ny, updated in
 * place).  Returns 0, or -1 when scratch memory cannot be allocated. */
int fv_ssprk3_steps(const fv_grid* G, const fv_coeffs* co, double* q0, double* q1, double* q2, double dt,
                    int nsteps) {
  const long n = (long)G->nx * G->ny;
  const int nq = co->nq;
  double* buf = (double*)malloc(sizeof(double) * (size_t)n * (6 * nq + 4 + 12));
  if (!buf) return -1;
  double* work = buf;
  double* st = buf + (long)(6 * nq + 4) * n;
  double* Q[3] = {q0, q1, q2};
  double* U1[3] = {st, st + n, st + 2 * n};
  double* U2[3] = {st + 3 * n, st + 4 * n, st + 5 * n};
  double* L[3] = {st + 6 * n, st + 7 * n, st + 8 * n};
  double* F[3] = {st + 9 * n, st + 10 * n, st + 11 * n};
  for (int step = 0; step < nsteps; ++step) {
    /* u1 = Q + dt L(Q) */
    rhs(G, co, Q, L, work);
    for (int c = 0; c < 3; ++c)
#pragma omp parallel for schedule(static)
      for (long t = 0; t < n; ++t) U1[c][t] = Q[c][t] + dt * L[c][t];
    /* u2 = 3/4 Q + 1/4 (u1 + dt L(u1)) */
    rhs(G, co, U1, L, work);
    for (int c = 0; c < 3; ++c)
#pragma omp parallel for schedule(static)
      for (long t = 0; t < n; ++t) {
        F[c][t] = U1[c][t] + dt * L[c][t];
        U2[c][t] = 0.75 * Q[c][t] + 0.25 * F[c][t];
      }
    /* Q = 1/3 Q + 2/3 (u2 + dt L(u2)) */
    rhs(G, co, U2, L, work);
    for (int c = 0; c < 3; ++c)
#pragma omp parallel for schedule(static)
      for (long t = 0; t < n; ++t) {
        F[c][t] = U2[c][t] + dt * L[c][t];
        Q[c][t] = Q[c][t] / 3.0 + 2.0 / 3.0 * F[c][t];
      }
  }
  free(buf);
  return 0;
}
