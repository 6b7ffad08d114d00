// Device helpers shared by the full-grid and Tucker kernels.
#pragma once

#include <cmath>

#include "dvm_internal.h"

namespace dvm {

struct CellMacro {
  double n, u[3], T, q[3];
  bool bad;
};

// Macroparameters from raw moment sums taken about the reference velocity r
// (Section 2 definitions with R_g = 1/2, m = 1):
//   n = w S0, u = r + M / S0, T = (2/3) (E / S0 - |u - r|^2),
//   q_a = (w/2) sum (xi_a - u_a) |xi - u|^2 f expanded about r.
__host__ __device__ inline void macro_from_sums(const double *S, double w, CellMacro &m) {
  const double S0 = S[3];
  const double ut0 = S[4] / S0, ut1 = S[5] / S0, ut2 = S[6] / S0;
  const double S11 = S[7], S22 = S[8], S33 = S[9], S12 = S[10], S13 = S[11], S23 = S[12];
  const double Et = S11 + S22 + S33;
  const double uu = ut0 * ut0 + ut1 * ut1 + ut2 * ut2;
  const double um = ut0 * S[4] + ut1 * S[5] + ut2 * S[6];
  m.n = w * S0;
  m.u[0] = S[0] + ut0;
  m.u[1] = S[1] + ut1;
  m.u[2] = S[2] + ut2;
  m.T = (2.0 / 3.0) * (Et / S0 - uu);
  const double us[3] = {ut0, ut1, ut2};
  const double Sab[3][3] = {{S11, S12, S13}, {S12, S22, S23}, {S13, S23, S33}};
  for (int a = 0; a < 3; ++a) {
    const double su = Sab[a][0] * ut0 + Sab[a][1] * ut1 + Sab[a][2] * ut2;
    m.q[a] = 0.5 * w *
             (S[13 + a] - 2.0 * su + uu * S[4 + a] - us[a] * Et + 2.0 * us[a] * um -
              us[a] * uu * S0);
  }
  m.bad = !(m.n > 0.0) || !(m.T > 0.0) || !isfinite(m.n) || !isfinite(m.T);
}

// conserved moments U = (n, n u, sum w |xi|^2 f) from sums about r
__device__ inline void conserved_from_sums(const double *S, double w, double U[5]) {
  const double S0 = S[3];
  const double r0 = S[0], r1 = S[1], r2 = S[2];
  const double Et = S[7] + S[8] + S[9];
  U[0] = w * S0;
  U[1] = w * (S[4] + r0 * S0);
  U[2] = w * (S[5] + r1 * S0);
  U[3] = w * (S[6] + r2 * S0);
  U[4] = w * (Et + 2.0 * (r0 * S[4] + r1 * S[5] + r2 * S[6]) + (r0 * r0 + r1 * r1 + r2 * r2) * S0);
}


}  // namespace dvm
