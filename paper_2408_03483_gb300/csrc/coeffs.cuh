// Reconstruction coefficients of Sec. 2.3, computed on the host from their
// definition: the degree-k polynomial matching k+1 cell averages evaluated at
// a face (Step 1) or at a Gauss point (Step 2).  Coordinates in cell units,
// cell j = [-1/2, 1/2]; candidate r uses cells j-r .. j-r+k.
#pragma once

namespace ttfv {

struct ReconCoeffs {
  // Gauss-Legendre points (cell units, ascending) and weights summing to 1
  double delta2[2], w2[2];
  double delta3[3], w3[3];
  // Step 2, nq = 2 (Upwind3): C[m][r][l]
  double C2[2][2][2];
  // Step 2, nq = 3 (Upwind5/WENO5): C[m][r][l]
  double C3[3][3][3];
  // linear weights gamma_m (nq = 3, m = 0 and 2); m = 1 uses the split
  double gam3[3][3];
  double gp[3], gm[3], sp, sm;  // split of m = 1 (the centre point)
  // combined linear Step-2 stencils over offsets -k..k: nq=2 (3 taps), nq=3 (5 taps)
  double lin2[2][3];
  double lin3[3][5];
  // combined linear Step-1 stencils over offsets -2..2 ("-": right face)
  double up3_minus[5], up3_plus[5], up5_minus[5], up5_plus[5];
};

const ReconCoeffs& recon_coeffs();

// Coefficients the WENO cross evaluators take by value.
struct WenoConst {
  double C3[3][3][3];
  double gam3[3][3];
  double gp[3], gm[3], sp, sm;
};
WenoConst weno_const();

}  // namespace ttfv
