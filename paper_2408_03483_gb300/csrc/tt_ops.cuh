// TT-level operations shared by the solver, the cross and the C ABI.
#pragma once
#include <vector>

#include "tt_common.cuh"

namespace ttfv {

constexpr int kMaxStencilOut = 8;
constexpr int kMaxTaps = 10;

struct StencilOut {
  double* dst = nullptr;  // output core (column-major)
  long ld = 0;            // its leading dimension
  int row0 = 0;           // first output row (stacked blocks)
  int ntaps = 0;
  int shift[kMaxTaps] = {};
  int base[kMaxTaps] = {};  // input row offset of the tap's block
  double coef[kMaxTaps] = {};
};
struct StencilSet {
  int nout = 0;
  StencilOut out[kMaxStencilOut];
};

struct Term {
  double c;
  TT x;
};

struct RoundInfo {
  int rank;
  double err;    // discarded Frobenius norm (incl. range-finder residual)
  double norm;   // Frobenius norm of the input
  double resid;  // range-finder residual (0 on exact routes)
};

void stencil(Exec& ex, const StencilSet& st, const double* in, long ldin, int n, int r);
void khatri_rao(Exec& ex, const double* X, int r1, const double* Y, int r2, int n, double* Z);
template <typename Real>
void transpose(Exec& ex, const Real* X, int m, int n, long ldx, Real* Y, long ldy);
void set_identity(Exec& ex, double* I, int p);
void tt_concat(Exec& ex, const std::vector<Term>& terms, TT& out);
int total_rank(const std::vector<Term>& terms);
void tt_sum_norm(Exec& ex, const TT& X, double* out_dev);

RoundInfo round_full(Exec& ex, const double* Yf, int n1, int n2, double tol, int cap, TT& Y);
// Truncation tolerance actually applied under ex.precision (the FP32 form
// does not truncate below its own round-off).
double effective_tol(const Exec& ex, double tol);
RoundInfo round_cores(Exec& ex, const double* A, const double* B, int n1, int n2, int R, double tol, int cap,
                      TT& Y);
RoundInfo round_tt(Exec& ex, const TT& X, double tol, int cap, TT& Y);
RoundInfo round_sum(Exec& ex, const std::vector<Term>& terms, double tol, int cap, TT& Y);
RoundInfo round_hadamard(Exec& ex, const TT& X, const TT& Z, double tol, int cap, TT& Y);

// Taylor-series reciprocal (Algorithm 1); returns iterations, sets *noconv.
int reciprocal(Exec& ex, const TT& x, double tol, int cap, int max_iter, TT& y, bool* noconv);

// Cross interpolation (cross.cu)
struct CrossFn {
  int fn = 0;
  const TT* in = nullptr;
  int nin = 0;
  double prm[4] = {0, 0, 0, 0};
  // the call site's converged column pivots of the previous stage (read by
  // the learned start, rewritten on exit); null: no memory
  std::vector<int>* site = nullptr;
};
int cross(Exec& ex, const CrossFn& f, int n1, int n2, const TT& x0, double tol, int cap, int kick,
          int max_sweeps, unsigned seed, TT& y);

// Learned-pivot network (mlp.cu): features X (n2 x 12, ld n2) of the column
// mode of x0; scores s of m rows; gradients of the mean logistic loss into g
// (same shapes as the parameters) and the loss into *loss (device, may be
// null); one Adam step of the FP32 masters; top-k indices ascending.
constexpr int kMlpFeatures = 14;
constexpr int kMlpHidden = 256;
// prev: device array of the site's previous converged pivots (nprev entries)
void mlp_features(Exec& ex, const TT& x0, const int* prev, int nprev, float* X);
void mlp_features_host_prev(Exec& ex, const TT& x0, const std::vector<int>& prev, float* X);
void mlp_forward(Exec& ex, const MlpNet& net, const float* X, int m, float* s);
void mlp_grad(Exec& ex, const MlpNet& net, const float* X, const float* y, int m, const MlpNet& g, double* loss);
void mlp_adam(Exec& ex, const MlpNet& p, const MlpNet& g, const MlpNet& m1, const MlpNet& m2, int t, float lr);
void mlp_topk(Exec& ex, const float* s, int m, int k, int* idx);
void mlp_propose(Exec& ex, const MlpNet& net, const TT& x0, const std::vector<int>& prev, int k, int* idx);

// Training-data capture (fv.cu): features of x0's column mode with a 0/1
// label per index (1: in the converged column pivot set J).
void record_pivots(Exec& ex, const TT& x0, const std::vector<int>& prev, const std::vector<int>& J);

// Linear reconstruction on cores (fv.cu)
void recon_linear(Exec& ex, const TT& x, int direction, int scheme, TT& qm, TT& qp);

}  // namespace ttfv
