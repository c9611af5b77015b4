// Expensive stencil evaluations S(k) (Section 2: every stencil evaluation carries a
// cost parameter k; Section 4: k evaluations of sin added to the prescribed entry,
// k = kmax on every vertex or running linearly over the mesh).  For the red-black
// finite-difference sweep the diagonal entry of interior vertex p becomes
//   2d + 2^-20 sigma_k(p) / k,   sigma_k(p) = sum_{m=1..k} sin(m theta_p),
//   theta_p = idx_p 2^-20,
// idx_p the lexicographic index of p among the interior vertices (x fastest) and
// k(p) = kmax (uniform) or floor(kmax idx_p / N) (linear over the N interior vertices;
// k = 0 keeps the plain diagonal).  The update is u_p = (h^2 f_p + sum of neighbours)
// / diagonal, with a correctly rounded division.
#pragma once
#include <stdint.h>

#include "internal.h"

namespace stencil {

enum { COST_NONE = 0, COST_UNIFORM = 1, COST_LINEAR = 2 };

__device__ __forceinline__ double cost_diagonal(const Geo &q, int dim, int mode, int kmax, int64_t i, int64_t j,
                                                int64_t k) {
  const int64_t rowlen = q.nx - 1, plane = (q.nx - 1) * (q.ny - 1);
  const int64_t idx = (dim == 3 ? (k - 1) * plane : 0) + (j - 1) * rowlen + (i - 1);
  const int64_t N = plane * (dim == 3 ? q.nz - 1 : 1);
  const int64_t kk = mode == COST_UNIFORM ? kmax : (mode == COST_LINEAR ? (int64_t)kmax * idx / N : 0);
  double diag = 2.0 * dim;
  if (kk > 0) {
    const double theta = (double)idx * 0x1p-20;
    double sigma = 0.0;
    for (int64_t m = 1; m <= kk; ++m) sigma += sin((double)m * theta);
    diag += 0x1p-20 * (sigma / (double)kk);
  }
  return diag;
}

}  // namespace stencil
