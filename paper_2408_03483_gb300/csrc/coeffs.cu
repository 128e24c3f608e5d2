// Host computation of the reconstruction coefficients (Sec. 2.3.1-2.3.2).
// The printed tables of Sec. 2.3.2 are rational approximations; these are the
// exact values from the defining polynomial problems.
#include <cmath>

#include "coeffs.cuh"
#include "tt_common.cuh"

namespace ttfv {

// average of x^d over the unit cell centred at s
static double cell_moment(int s, int d) {
  const double a = s - 0.5, b = s + 0.5;
  return (std::pow(b, d + 1) - std::pow(a, d + 1)) / (d + 1);
}

// weights c_l with p(x) = sum_l c_l v_{cells[l]}; solves M^T c = e(x) with
// M[l][d] = cell_moment(cells[l], d) by Gaussian elimination, partial pivoting.
static void point_coeffs(const int* cells, int k1, double x, double* out) {
  double A[5][6];
  for (int d = 0; d < k1; ++d) {       // row d of M^T
    for (int l = 0; l < k1; ++l) A[d][l] = cell_moment(cells[l], d);
    A[d][k1] = std::pow(x, d);
  }
  for (int c = 0; c < k1; ++c) {
    int p = c;
    for (int i = c + 1; i < k1; ++i)
      if (std::fabs(A[i][c]) > std::fabs(A[p][c])) p = i;
    if (p != c)
      for (int j = 0; j <= k1; ++j) std::swap(A[c][j], A[p][j]);
    for (int i = 0; i < k1; ++i) {
      if (i == c) continue;
      const double f = A[i][c] / A[c][c];
      for (int j = c; j <= k1; ++j) A[i][j] -= f * A[c][j];
    }
  }
  for (int l = 0; l < k1; ++l) out[l] = A[l][k1] / A[l][l];
}

static ReconCoeffs build() {
  ReconCoeffs R{};
  const double d2 = 1.0 / (2.0 * std::sqrt(3.0));
  R.delta2[0] = -d2;
  R.delta2[1] = d2;
  R.w2[0] = R.w2[1] = 0.5;
  const double d3 = std::sqrt(15.0) / 10.0;
  R.delta3[0] = -d3;
  R.delta3[1] = 0.0;
  R.delta3[2] = d3;
  R.w3[0] = R.w3[2] = 5.0 / 18.0;
  R.w3[1] = 8.0 / 18.0;
  // Step 2 candidates
  for (int m = 0; m < 2; ++m)
    for (int r = 0; r < 2; ++r) {
      int cells[2] = {-r, -r + 1};
      point_coeffs(cells, 2, R.delta2[m], R.C2[m][r]);
    }
  for (int m = 0; m < 3; ++m)
    for (int r = 0; r < 3; ++r) {
      int cells[3] = {-r, -r + 1, -r + 2};
      point_coeffs(cells, 3, R.delta3[m], R.C3[m][r]);
    }
  // gamma at the outer points: the unique weights that make the three 3-cell
  // values combine into the 5-cell value; offsets -2 and +2 are reached by one
  // candidate each, offset -1 then fixes the middle weight.
  for (int m = 0; m < 3; m += 2) {
    int cells5[5] = {-2, -1, 0, 1, 2};
    double c5[5];
    point_coeffs(cells5, 5, R.delta3[m], c5);
    const double g2 = c5[0] / R.C3[m][2][0];   // r=2 covers -2..0
    const double g0 = c5[4] / R.C3[m][0][2];   // r=0 covers 0..2
    const double g1 = (c5[1] - g2 * R.C3[m][2][1]) / R.C3[m][1][0];
    R.gam3[m][0] = g0;
    R.gam3[m][1] = g1;
    R.gam3[m][2] = g2;
  }
  // centre point: the split weights printed in Sec. 2.3.2 (exact)
  R.gp[0] = 9.0 / 214.0;
  R.gp[1] = 98.0 / 107.0;
  R.gp[2] = 9.0 / 214.0;
  R.gm[0] = 9.0 / 67.0;
  R.gm[1] = 49.0 / 67.0;
  R.gm[2] = 9.0 / 67.0;
  R.sp = 107.0 / 40.0;
  R.sm = 67.0 / 40.0;
  for (int r = 0; r < 3; ++r) R.gam3[1][r] = R.sp * R.gp[r] - R.sm * R.gm[r];
  // combined linear stencils
  for (int m = 0; m < 2; ++m) {
    for (int t = 0; t < 3; ++t) R.lin2[m][t] = 0.0;
    for (int r = 0; r < 2; ++r)
      for (int l = 0; l < 2; ++l) R.lin2[m][(-r + l) + 1] += 0.5 * R.C2[m][r][l];
  }
  for (int m = 0; m < 3; ++m) {
    for (int t = 0; t < 5; ++t) R.lin3[m][t] = 0.0;
    for (int r = 0; r < 3; ++r)
      for (int l = 0; l < 3; ++l) R.lin3[m][(-r + l) + 2] += R.gam3[m][r] * R.C3[m][r][l];
  }
  // Step 1 (printed candidates and ideal weights, "-" side = right face)
  const double up3[5] = {0.0, -1.0 / 6.0, 5.0 / 6.0, 1.0 / 3.0, 0.0};
  const double up5[5] = {2.0 / 60.0, -13.0 / 60.0, 47.0 / 60.0, 27.0 / 60.0, -3.0 / 60.0};
  for (int t = 0; t < 5; ++t) {
    R.up3_minus[t] = up3[t];
    R.up3_plus[t] = up3[4 - t];
    R.up5_minus[t] = up5[t];
    R.up5_plus[t] = up5[4 - t];
  }
  return R;
}

const ReconCoeffs& recon_coeffs() {
  static ReconCoeffs R = build();
  return R;
}

WenoConst weno_const() {
  const ReconCoeffs& R = recon_coeffs();
  WenoConst w{};
  for (int m = 0; m < 3; ++m)
    for (int r = 0; r < 3; ++r) {
      w.gam3[m][r] = R.gam3[m][r];
      for (int l = 0; l < 3; ++l) w.C3[m][r][l] = R.C3[m][r][l];
    }
  for (int r = 0; r < 3; ++r) {
    w.gp[r] = R.gp[r];
    w.gm[r] = R.gm[r];
  }
  w.sp = R.sp;
  w.sm = R.sm;
  return w;
}

}  // namespace ttfv
