// Derivative of one entry of the Slater-Koster sp block with respect to the bond vector (device code
// shared by the force kernels).
#pragma once

#include <math.h>

namespace mka {

// d/dd of entry [row][col] of the two-centre block for displacement d (s, px, py, pz order):
//   [s][s] = ss s(r), [s][p_k] = c_k sp s(r), [p_k][s] = -[s][p_k],
//   [p_k][p_m] = c_k c_m (pps - ppp) s(r) + delta_km ppp s(r), s(r) = exp(-2 (r/d0 - 1)), c = d / r.
__device__ __forceinline__ void sk_entry_grad(const double d[3], const double V[4], double d0, int row, int col, double out[3]) {
  const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  const double ir = 1.0 / r;
  const double c[3] = {d[0] * ir, d[1] * ir, d[2] * ir};
  const double s = exp(-2.0 * (r / d0 - 1.0));
  const double sr = -(2.0 / d0) * s;      // ds/dr
  for (int l = 0; l < 3; ++l) {
    const double ds = sr * c[l];
    double g;
    if (row == 0 && col == 0) {
      g = V[0] * ds;
    } else if (row == 0 || col == 0) {
      const int k = (row == 0 ? col : row) - 1;
      const double dck = ((k == l ? 1.0 : 0.0) - c[k] * c[l]) * ir;
      g = V[1] * (dck * s + c[k] * ds);
      if (col == 0) g = -g;
    } else {
      const int k = row - 1, m = col - 1;
      const double dck = ((k == l ? 1.0 : 0.0) - c[k] * c[l]) * ir;
      const double dcm = ((m == l ? 1.0 : 0.0) - c[m] * c[l]) * ir;
      g = (V[2] - V[3]) * ((dck * c[m] + c[k] * dcm) * s + c[k] * c[m] * ds) + (k == m ? V[3] * ds : 0.0);
    }
    out[l] = g;
  }
}

}  // namespace mka
