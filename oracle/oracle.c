/*
 * Oracle for Hazelwood & Weinzierl, "Coloured and task-based stencil codes"
 * (arXiv:1810.04033): plain FP64 C, slow on purpose, written so that each function
 * can be checked against the paper and the mathematics by eye.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU-baseline
 * leg of the benchmark.  The GPU library never calls it and shares nothing with it.
 *
 * Compile with -ffp-contract=off so that no multiply-add is fused and the x86 and Arm
 * builds produce identical bits.
 *
 * Parity status per function (what pins it; the pins live in tests/):
 *   oracle_q1_element_matrix  pinned: its 2D assembly reproduces the paper's printed
 *                             9-point stencil (Fig. 1); 3D row sums, symmetry.
 *   oracle_apply_elementwise  pinned: equals a Kronecker-product assembly of the global
 *                             matrix; annihilates constants/linears; exact -Laplacian
 *                             on cubic polynomials; symbol on sine modes.
 *   oracle_apply_stencil      pinned: as above plus equality with the element form.
 *   oracle_gs_coloured        pinned: brute-force dense-matrix Gauss-Seidel in colour
 *                             order; order-independence inside a colour; convergence
 *                             to the closed-form discrete solution.
 *   oracle_gs_coloured_f32    pinned: FP32 sweep vs FP64 sweep within FP32 rounding;
 *                             float-rounded brute force on tiny grids.
 *   oracle_gs_coloured_bf16   pinned: bf16 rounding helpers against torch's bf16
 *                             casts; sweep vs FP32 sweep within bf16 rounding.
 *   oracle_jacobi             pinned: closed-form eigenmode damping factor; dense
 *                             brute force.
 *   oracle_residual           pinned: dense brute force; zero at the discrete solution;
 *                             exact rational arithmetic on tiny grids, within a
 *                             forward error bound.
 *   oracle_residual_ld        pinned: exact rational arithmetic on tiny grids.
 *   oracle_ir_solve           pinned: converges to the closed-form discrete solution of
 *                             the manufactured problem; FP64 inner equals plain GS.
 *   oracle_mg_*               pinned: Galerkin identity R A_h P = A_2h on random
 *                             coarse vectors (nested grids); P reproduces d-linear
 *                             functions (nested and not); R is (n_c/n)^d P^T (adjoint
 *                             identity); the solve reaches the closed-form discrete
 *                             solution for even and odd n; V-cycle contraction.
 *   oracle_fd_*               pinned: the 5-point stencil printed in Fig. 1 (golden
 *                             file); dense Kronecker assembly; exactness on cubic
 *                             polynomials; sine-mode symbol and closed-form solution;
 *                             red-black GS = dense GS in Algorithm 1's colour order.
 *   oracle_*cost*             pinned: mode 0 equals the plain red-black sweep; the
 *                             linear k pattern (0 on the first 1/kmax of the interior);
 *                             the sweep equals a dense GS on the matrix with the
 *                             perturbed diagonal; sigma_k against the closed form
 *                             sin(k t/2) sin((k+1) t/2) / sin(t/2).
 *   oracle_patch_*            equal sizes pinned: the iteration converges to the dense
 *                             solution of the global system on the collapsed grid of
 *                             the patches' interiors (faces, edges and corners of the
 *                             halo alike); a single patch with zero neighbours equals a
 *                             plain Dirichlet GS; equal-size neighbours copy the first
 *                             interior layer.  Uneven sizes: parity unpinned beyond the
 *                             nearest-index and tie checks (the halo rule is a reading,
 *                             the paper is silent on it).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- grid helpers */

static int64_t nz_cells(int dim, const int64_t *n) { return dim == 3 ? n[2] : 0; }

static int64_t num_points(int dim, const int64_t *n) {
  return (n[0] + 1) * (n[1] + 1) * (nz_cells(dim, n) + 1);
}

static int64_t vidx(const int64_t *n, int64_t i, int64_t j, int64_t k) {
  return (k * (n[1] + 1) + j) * (n[0] + 1) + i;
}

static int is_interior(int dim, const int64_t *n, int64_t i, int64_t j, int64_t k) {
  if (i <= 0 || i >= n[0] || j <= 0 || j >= n[1]) return 0;
  if (dim == 3 && (k <= 0 || k >= n[2])) return 0;
  return 1;
}

static int colour_of(int64_t i, int64_t j, int64_t k) {
  return (int)((i & 1) + 2 * (j & 1) + 4 * (k & 1));
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
  omp_set_num_threads(nthreads > 0 ? nthreads : 1);
#else
  (void)nthreads;
#endif
}

/* ------------------------------------------------ element matrix and stencil */

void oracle_q1_element_matrix(int dim, double h, double *Ke) {
  /* 1D element stiffness and mass on [0,h] for the two linear hat functions. */
  const double a1[2][2] = {{1.0 / h, -1.0 / h}, {-1.0 / h, 1.0 / h}};
  const double m1[2][2] = {{2.0 * h / 6.0, h / 6.0}, {h / 6.0, 2.0 * h / 6.0}};
  const int nv = 1 << dim;
  for (int v = 0; v < nv; ++v) {
    for (int w = 0; w < nv; ++w) {
      /* grad.grad integrates to a sum over axes of (stiffness on that axis) times
         (mass on every other axis). */
      double sum = 0.0;
      for (int axis = 0; axis < dim; ++axis) {
        double prod = 1.0;
        for (int b = 0; b < dim; ++b) {
          const int vb = (v >> b) & 1, wb = (w >> b) & 1;
          prod *= (b == axis) ? a1[vb][wb] : m1[vb][wb];
        }
        sum += prod;
      }
      Ke[v * nv + w] = sum;
    }
  }
}

double oracle_stencil_weight(int dim, int dx, int dy, int dz) {
  /* Assembled Q1 stencil, h-free.  A vertex pair that differs in m coordinates is
     shared by 2^(d-m) cells; summing the element entries gives these weights. */
  const int m = (dx != 0) + (dy != 0) + (dim == 3 ? (dz != 0) : 0);
  if (dim == 2) {
    if (m == 0) return 8.0 / 3.0;
    return -1.0 / 3.0; /* Fig. 1, right: all eight neighbours -1/3 */
  }
  if (m == 0) return 8.0 / 3.0;
  if (m == 1) return 0.0;
  if (m == 2) return -1.0 / 6.0;
  return -1.0 / 12.0;
}

/* ------------------------------------------------------------------- applies */

void oracle_apply_elementwise(int dim, const int64_t *n, double h,
                              const double *u, double *y, int nthreads) {
  const int nv = 1 << dim;
  double Ke[64];
  oracle_q1_element_matrix(dim, h, Ke);
  const int64_t np = num_points(dim, n);
  const int64_t ncz = dim == 3 ? n[2] : 1;
  const int64_t nrows = ncz * n[1];
  set_threads(nthreads);
  for (int64_t p = 0; p < np; ++p) y[p] = 0.0;

  /* Colour passes over the cells: cells of one colour share no vertex, so the
     scatter inside one pass is race free. */
  for (int c = 0; c < nv; ++c) {
#pragma omp parallel for schedule(static) if (nthreads > 1)
    for (int64_t row = 0; row < nrows; ++row) {
      const int64_t ck = dim == 3 ? row / n[1] : 0, cj = row % n[1];
      for (int64_t ci = 0; ci < n[0]; ++ci) {
        if (colour_of(ci, cj, ck) != c) continue;
        int64_t vert[8];
        for (int v = 0; v < nv; ++v)
          vert[v] = vidx(n, ci + (v & 1), cj + ((v >> 1) & 1),
                         dim == 3 ? ck + ((v >> 2) & 1) : 0);
        for (int v = 0; v < nv; ++v) {
          double acc = 0.0;
          for (int w = 0; w < nv; ++w) acc += Ke[v * nv + w] * u[vert[w]];
          y[vert[v]] += acc;
        }
      }
    }
  }
  /* Divide by the lumped mass h^d; boundary rows are not equations. */
  const double hd = dim == 3 ? h * h * h : h * h;
  const int64_t nzc = nz_cells(dim, n);
  for (int64_t k = 0; k <= nzc; ++k)
    for (int64_t j = 0; j <= n[1]; ++j)
      for (int64_t i = 0; i <= n[0]; ++i) {
        const int64_t p = vidx(n, i, j, k);
        y[p] = is_interior(dim, n, i, j, k) ? y[p] / hd : 0.0;
      }
}

/* (S u)_i over all 3^d offsets, dz outer, then dy, then dx, each from -1 to 1.
   skip_centre leaves the diagonal term out. */
static double stencil_sum(int dim, const int64_t *n, const double *u, int64_t i,
                          int64_t j, int64_t k, int skip_centre) {
  double acc = 0.0;
  const int zlo = dim == 3 ? -1 : 0, zhi = dim == 3 ? 1 : 0;
  for (int dz = zlo; dz <= zhi; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (skip_centre && dx == 0 && dy == 0 && dz == 0) continue;
        acc += oracle_stencil_weight(dim, dx, dy, dz) * u[vidx(n, i + dx, j + dy, k + dz)];
      }
  return acc;
}

void oracle_apply_stencil(int dim, const int64_t *n, double h, const double *u,
                          double *y, int nthreads) {
  const int64_t nzc = nz_cells(dim, n);
  const double h2 = h * h;
  set_threads(nthreads);
#pragma omp parallel for schedule(static) if (nthreads > 1)
  for (int64_t k = 0; k <= nzc; ++k)
    for (int64_t j = 0; j <= n[1]; ++j)
      for (int64_t i = 0; i <= n[0]; ++i) {
        const int64_t p = vidx(n, i, j, k);
        y[p] = is_interior(dim, n, i, j, k) ? stencil_sum(dim, n, u, i, j, k, 0) / h2 : 0.0;
      }
}

/* -------------------------------------------------------- coloured Gauss-Seidel */

void oracle_gs_coloured(int dim, const int64_t *n, double h, double *u,
                        const double *f, int sweeps, int nthreads) {
  const int ncol = 1 << dim;
  const int64_t klo = dim == 3 ? 1 : 0;
  const int64_t nrows = (dim == 3 ? n[2] - 1 : 1) * (n[1] - 1);
  const double h2 = h * h;
  const double w0 = oracle_stencil_weight(dim, 0, 0, 0);
  set_threads(nthreads);
  for (int s = 0; s < sweeps; ++s) {
    for (int c = 0; c < ncol; ++c) {
      /* One colour pass over the interior rows (k, j), lexicographic: its updates
         read no vertex of the same colour, so the rows may be split across threads
         (the paper's parallel for over the outer loop). */
#pragma omp parallel for schedule(static) if (nthreads > 1)
      for (int64_t row = 0; row < nrows; ++row) {
        const int64_t k = klo + row / (n[1] - 1), j = 1 + row % (n[1] - 1);
        for (int64_t i = 1; i < n[0]; ++i) {
          if (colour_of(i, j, k) != c) continue;
          /* in-situ update: u_i <- (h^2 f_i - sum_{j != i} s_ij u_j) / s_ii */
          const double off = stencil_sum(dim, n, u, i, j, k, 1);
          const int64_t p = vidx(n, i, j, k);
          u[p] = (h2 * f[p] - off) / w0;
        }
      }
    }
  }
}

void oracle_gs_coloured_f32(int dim, const int64_t *n, double h, float *u,
                            const float *f, int sweeps) {
  const int ncol = 1 << dim;
  const int64_t nzc = nz_cells(dim, n);
  const int64_t klo = dim == 3 ? 1 : 0, khi = dim == 3 ? nzc - 1 : 0;
  const float h2 = (float)(h * h);
  const float w0 = (float)oracle_stencil_weight(dim, 0, 0, 0);
  const int zlo = dim == 3 ? -1 : 0, zhi = dim == 3 ? 1 : 0;
  for (int s = 0; s < sweeps; ++s)
    for (int c = 0; c < ncol; ++c)
      for (int64_t k = klo; k <= khi; ++k)
        for (int64_t j = 1; j < n[1]; ++j)
          for (int64_t i = 1; i < n[0]; ++i) {
            if (colour_of(i, j, k) != c) continue;
            float off = 0.0f;
            for (int dz = zlo; dz <= zhi; ++dz)
              for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                  if (dx == 0 && dy == 0 && dz == 0) continue;
                  off += (float)oracle_stencil_weight(dim, dx, dy, dz) *
                         u[vidx(n, i + dx, j + dy, k + dz)];
                }
            const int64_t p = vidx(n, i, j, k);
            u[p] = (h2 * f[p] - off) / w0;
          }
}

uint16_t oracle_f32_to_bf16(float x) {
  /* bf16 keeps the upper 16 bits of the binary32 pattern; round to nearest, ties to
     even, by adding half an ulp of the kept part (minus one when the kept part is
     even) before truncating.  NaN stays NaN. */
  uint32_t b;
  memcpy(&b, &x, sizeof b);
  if ((b & 0x7f800000u) == 0x7f800000u && (b & 0x007fffffu) != 0)
    return (uint16_t)((b >> 16) | 0x0040u);
  const uint32_t lsb = (b >> 16) & 1u;
  b += 0x7fffu + lsb;
  return (uint16_t)(b >> 16);
}

float oracle_bf16_to_f32(uint16_t v) {
  const uint32_t b = (uint32_t)v << 16;
  float x;
  memcpy(&x, &b, sizeof x);
  return x;
}

void oracle_gs_coloured_bf16(int dim, const int64_t *n, double h, uint16_t *u,
                             const uint16_t *f, int sweeps) {
  const int ncol = 1 << dim;
  const int64_t nzc = nz_cells(dim, n);
  const int64_t klo = dim == 3 ? 1 : 0, khi = dim == 3 ? nzc - 1 : 0;
  const float h2 = (float)(h * h);
  const float w0 = (float)oracle_stencil_weight(dim, 0, 0, 0);
  const int zlo = dim == 3 ? -1 : 0, zhi = dim == 3 ? 1 : 0;
  for (int s = 0; s < sweeps; ++s)
    for (int c = 0; c < ncol; ++c)
      for (int64_t k = klo; k <= khi; ++k)
        for (int64_t j = 1; j < n[1]; ++j)
          for (int64_t i = 1; i < n[0]; ++i) {
            if (colour_of(i, j, k) != c) continue;
            float off = 0.0f;
            for (int dz = zlo; dz <= zhi; ++dz)
              for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                  if (dx == 0 && dy == 0 && dz == 0) continue;
                  off += (float)oracle_stencil_weight(dim, dx, dy, dz) *
                         oracle_bf16_to_f32(u[vidx(n, i + dx, j + dy, k + dz)]);
                }
            const int64_t p = vidx(n, i, j, k);
            u[p] = oracle_f32_to_bf16((h2 * oracle_bf16_to_f32(f[p]) - off) / w0);
          }
}

/* --------------------------------------------------------------------- Jacobi */

void oracle_jacobi(int dim, const int64_t *n, double h, double *u,
                   const double *f, double *work, double omega, int sweeps,
                   int nthreads) {
  const int64_t nzc = nz_cells(dim, n);
  const int64_t np = num_points(dim, n);
  const double h2 = h * h;
  const double w0 = oracle_stencil_weight(dim, 0, 0, 0);
  set_threads(nthreads);
  for (int s = 0; s < sweeps; ++s) {
    /* every new value is computed from the unchanged old array */
#pragma omp parallel for schedule(static) if (nthreads > 1)
    for (int64_t k = 0; k <= nzc; ++k)
      for (int64_t j = 0; j <= n[1]; ++j)
        for (int64_t i = 0; i <= n[0]; ++i) {
          const int64_t p = vidx(n, i, j, k);
          if (!is_interior(dim, n, i, j, k)) {
            work[p] = u[p];
            continue;
          }
          /* u + omega * D^-1 (f - A u), D = s_ii / h^2 */
          const double res = h2 * f[p] - stencil_sum(dim, n, u, i, j, k, 0);
          work[p] = u[p] + omega * (res / w0);
        }
    memcpy(u, work, (size_t)np * sizeof(double));
  }
}

/* ------------------------------------------------------------------- residual */

void oracle_residual(int dim, const int64_t *n, double h, const double *u,
                     const double *f, double *r, double *norms2, int nthreads) {
  const int64_t nzc = nz_cells(dim, n);
  const int64_t np = num_points(dim, n);
  const double h2 = h * h;
  double *res = r ? r : (double *)malloc((size_t)np * sizeof(double));
  set_threads(nthreads);
  /* r_i = f_i - (S u)_i / h^2, independent per vertex */
#pragma omp parallel for schedule(static) if (nthreads > 1)
  for (int64_t k = 0; k <= nzc; ++k)
    for (int64_t j = 0; j <= n[1]; ++j)
      for (int64_t i = 0; i <= n[0]; ++i) {
        const int64_t p = vidx(n, i, j, k);
        res[p] = is_interior(dim, n, i, j, k)
                     ? f[p] - stencil_sum(dim, n, u, i, j, k, 0) / h2
                     : 0.0;
      }
  /* both sums in lexicographic order over interior vertices, one thread */
  double rr = 0.0, ff = 0.0;
  for (int64_t k = 0; k <= nzc; ++k)
    for (int64_t j = 0; j <= n[1]; ++j)
      for (int64_t i = 0; i <= n[0]; ++i) {
        if (!is_interior(dim, n, i, j, k)) continue;
        const int64_t p = vidx(n, i, j, k);
        rr += res[p] * res[p];
        ff += f[p] * f[p];
      }
  norms2[0] = rr;
  norms2[1] = ff;
  if (!r) free(res);
}

/* The same norms in long double throughout (stencil weights as long double quotients,
 * products, the division by h^2 and both sums), from the same FP64 inputs: a near-exact
 * value against which the rounding of oracle_residual itself can be bounded (the FP64
 * norms must lie within a standard forward error bound of these).  One thread,
 * lexicographic order; norms2_ld receives the two sums rounded to double. */
static long double stencil_weight_ld(int dim, int dx, int dy, int dz) {
  const int m = (dx != 0) + (dy != 0) + (dim == 3 ? (dz != 0) : 0);
  if (m == 0) return 8.0L / 3.0L;
  if (dim == 2) return -1.0L / 3.0L;
  if (m == 1) return 0.0L;
  if (m == 2) return -1.0L / 6.0L;
  return -1.0L / 12.0L;
}

void oracle_residual_ld(int dim, const int64_t *n, double h, const double *u,
                        const double *f, double *norms2_ld) {
  const int64_t nzc = nz_cells(dim, n);
  const long double h2 = (long double)h * (long double)h;
  const int zlo = dim == 3 ? -1 : 0, zhi = dim == 3 ? 1 : 0;
  long double rr = 0.0L, ff = 0.0L;
  for (int64_t k = 0; k <= nzc; ++k)
    for (int64_t j = 0; j <= n[1]; ++j)
      for (int64_t i = 0; i <= n[0]; ++i) {
        if (!is_interior(dim, n, i, j, k)) continue;
        long double s = 0.0L;
        for (int dz = zlo; dz <= zhi; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx)
              s += stencil_weight_ld(dim, dx, dy, dz) *
                   (long double)u[vidx(n, i + dx, j + dy, k + dz)];
        const long double fi = (long double)f[vidx(n, i, j, k)];
        const long double r = fi - s / h2;
        rr += r * r;
        ff += fi * fi;
      }
  norms2_ld[0] = (double)rr;
  norms2_ld[1] = (double)ff;
}

/* ------------------------------------------------------ iterative refinement */

/* Steps of one outer iteration, starting from the FP64 iterate x:
 *   1. r = f - A x in FP64 and rho = ||r|| / ||f||; stop when rho <= tol;
 *   2. round r to the inner storage type (FP32: round to nearest; bf16: to FP32
 *      first, then to bf16 with ties to even);
 *   3. e = 0, then `inner_sweeps` coloured GS sweeps on A e = r in that precision;
 *   4. x += e, widened exactly to FP64, on interior vertices. */
int oracle_ir_solve(int dim, const int64_t *n, double h, double *x,
                    const double *f, double tol, int max_outer, int inner_sweeps,
                    int inner_prec, double *relres, double *x_hist,
                    int *converged) {
  const int64_t np = num_points(dim, n);
  double *r = (double *)malloc((size_t)np * sizeof(double));
  double *e64 = (double *)malloc((size_t)np * sizeof(double));
  float *r32 = (float *)malloc((size_t)np * sizeof(float));
  float *e32 = (float *)malloc((size_t)np * sizeof(float));
  uint16_t *r16 = (uint16_t *)malloc((size_t)np * sizeof(uint16_t));
  uint16_t *e16 = (uint16_t *)malloc((size_t)np * sizeof(uint16_t));
  int k = 0;
  *converged = 0;
  for (;;) {
    double nrm[2];
    oracle_residual(dim, n, h, x, f, r, nrm, 1);
    const double rho = sqrt(nrm[0]) / sqrt(nrm[1]);
    if (relres) relres[k] = rho;
    if (rho <= tol) {
      *converged = 1;
      break;
    }
    if (k >= max_outer) break;
    for (int64_t p = 0; p < np; ++p) {
      if (inner_prec == 0) {
        e64[p] = 0.0;
      } else if (inner_prec == 1) {
        r32[p] = (float)r[p];
        e32[p] = 0.0f;
      } else {
        r16[p] = oracle_f32_to_bf16((float)r[p]);
        e16[p] = 0;
      }
    }
    if (inner_prec == 0)
      oracle_gs_coloured(dim, n, h, e64, r, inner_sweeps, 1);
    else if (inner_prec == 1)
      oracle_gs_coloured_f32(dim, n, h, e32, r32, inner_sweeps);
    else
      oracle_gs_coloured_bf16(dim, n, h, e16, r16, inner_sweeps);
    const int64_t nzc = nz_cells(dim, n);
    for (int64_t kk = 0; kk <= nzc; ++kk)
      for (int64_t j = 0; j <= n[1]; ++j)
        for (int64_t i = 0; i <= n[0]; ++i) {
          if (!is_interior(dim, n, i, j, kk)) continue;
          const int64_t p = vidx(n, i, j, kk);
          const double e = inner_prec == 0   ? e64[p]
                           : inner_prec == 1 ? (double)e32[p]
                                             : (double)oracle_bf16_to_f32(e16[p]);
          x[p] += e;
        }
    if (x_hist) memcpy(x_hist + (size_t)k * (size_t)np, x, (size_t)np * sizeof(double));
    ++k;
  }
  free(r);
  free(e64);
  free(r32);
  free(e32);
  free(r16);
  free(e16);
  return k;
}

/* ----------------------------------------------------------- patch lattices */

/* Halo rule (a reading; the paper only says that regular patches sit inside a
 * block-structured mesh, Section 2).  Patch p at lattice position P covers
 * [P, P+1)^3 in lattice units with n_p cells per edge.  Each vertex of p whose index
 * is 0 or n_p on some axis is refilled as follows: the outward direction d has
 * d_a = -1 where the index is 0, +1 where it is n_p, 0 otherwise; if P + d lies
 * outside the lattice the value is 0; otherwise q = P + d and, per axis, the
 * vertex of q nearest to the halo vertex's position (ties to the lower index),
 * clamped to q's interior range [1, n_q - 1], supplies the value. */
void oracle_patch_halo_fill(const int32_t *lat, const int32_t *np,
                            const int64_t *off, double *u_all) {
  const int64_t npatch = (int64_t)lat[0] * lat[1] * lat[2];
  for (int64_t p = 0; p < npatch; ++p) {
    const int64_t P[3] = {p % lat[0], (p / lat[0]) % lat[1], p / ((int64_t)lat[0] * lat[1])};
    const int64_t n = np[p];
    const int64_t nn[3] = {n, n, n};
    double *u = u_all + off[p];
    for (int64_t k = 0; k <= n; ++k)
      for (int64_t j = 0; j <= n; ++j)
        for (int64_t i = 0; i <= n; ++i) {
          const int64_t idx[3] = {i, j, k};
          int d[3], on_shell = 0, outside = 0;
          int64_t Q[3];
          for (int a = 0; a < 3; ++a) {
            d[a] = idx[a] == 0 ? -1 : (idx[a] == n ? 1 : 0);
            on_shell |= d[a] != 0;
            Q[a] = P[a] + d[a];
            outside |= (Q[a] < 0 || Q[a] >= lat[a]);
          }
          if (!on_shell) continue;
          const int64_t dst = vidx(nn, i, j, k);
          if (outside) {
            u[dst] = 0.0;
            continue;
          }
          const int64_t q = Q[0] + lat[0] * (Q[1] + (int64_t)lat[1] * Q[2]);
          const int64_t m = np[q];
          int64_t iq[3];
          for (int a = 0; a < 3; ++a) {
            /* position in q's local cells = (idx - d*n) * m / n; nearest index with
               ties to the lower one = floor((2*num + n - 1) / (2n)), num >= 0 */
            const int64_t num = (idx[a] - d[a] * n) * m;
            int64_t t = (2 * num + n - 1) / (2 * n);
            if (t < 1) t = 1;
            if (t > m - 1) t = m - 1;
            iq[a] = t;
          }
          const int64_t mm[3] = {m, m, m};
          u[dst] = u_all[off[q] + vidx(mm, iq[0], iq[1], iq[2])];
        }
  }
}

void oracle_patch_smooth(const int32_t *lat, const int32_t *np,
                         const int64_t *off, double *u_all, const double *f_all,
                         int sweeps, int nthreads) {
  const int64_t npatch = (int64_t)lat[0] * lat[1] * lat[2];
  for (int s = 0; s < sweeps; ++s) {
    oracle_patch_halo_fill(lat, np, off, u_all);
    for (int64_t p = 0; p < npatch; ++p) {
      const int64_t nn[3] = {np[p], np[p], np[p]};
      oracle_gs_coloured(3, nn, 1.0 / (double)np[p], u_all + off[p], f_all + off[p], 1,
                         nthreads);
    }
  }
}

/* ------------------------------------------------------ geometric multigrid */

/* The paper names smoothers of matrix-free multigrid codes as the use of its sweeps
 * (Section 1).  A standard vertex-centred V-cycle with the coloured Gauss-Seidel as
 * smoother, written out from its textbook definition:
 *   coarse grid: n_c = n / 2 cells per axis when every n[a] is even (every second
 *   vertex), otherwise, for a grid with the same n on every axis, n_c = ceil(n / 2) on
 *   every axis (coarse vertices not nested in the fine ones); the coarse cells are
 *   cubes of side h_c = h n / n_c.  Grids are coarsened while every n[a] >= 4.
 *   prolongation P: d-linear interpolation of the coarse values at the fine vertex
 *   positions x_i = i / n (in units of the domain side), coarse vertices at I / n_c;
 *   restriction R = (n_c / n)^d P^T (full weighting when nested), which for the Q1
 *   operator A = S / h^2 gives the Galerkin identity R A_h P = A_2h in the nested case;
 *   V-cycle(u, f): `pre` sweeps; r = f - A u; e_c = V-cycle(0, R r) on the coarse grid
 *   (or `coarse_sweeps` sweeps on the coarsest grid); u += P e_c; `post` sweeps. */

/* Coarse grid of n (returns 0 when n is the coarsest grid). */
static int mg_coarsen(int dim, const int64_t *n, int64_t *nc) {
  int all_even = 1, all_equal = 1;
  for (int a = 0; a < dim; ++a) {
    if (n[a] < 4) return 0;
    if (n[a] % 2) all_even = 0;
    if (n[a] != n[0]) all_equal = 0;
  }
  if (!all_even && !all_equal) return 0;
  for (int a = 0; a < 3; ++a) nc[a] = a < dim ? (n[a] + 1) / 2 : 0;
  return 1;
}

int oracle_mg_levels(int dim, const int64_t *n, int max_levels) {
  int64_t m[3] = {n[0], n[1], dim == 3 ? n[2] : 0}, c[3];
  int L = 1;
  while (L < max_levels && mg_coarsen(dim, m, c)) {
    for (int a = 0; a < 3; ++a) m[a] = c[a];
    ++L;
  }
  return L;
}

/* 1D interpolation weight of coarse vertex I (of nc cells) at fine vertex i (of nf
 * cells): 1 - |i nc / nf - I| where positive, else 0 (exact integer arithmetic for the
 * distance, one division). */
static double interp_w(int64_t i, int64_t nf, int64_t I, int64_t nc) {
  int64_t d = i * nc - I * nf;
  if (d < 0) d = -d;
  return d >= nf ? 0.0 : (double)(nf - d) / (double)nf;
}

/* Fine indices i in [*lo, *hi] that can see coarse vertex I (|i nc - I nf| < nf). */
static void fine_range(int64_t I, int64_t nf, int64_t nc, int64_t *lo, int64_t *hi) {
  int64_t a = ((I - 1) * nf) / nc, b = ((I + 1) * nf + nc - 1) / nc;
  *lo = a < 0 ? 0 : a;
  *hi = b > nf ? nf : b;
}

void oracle_mg_restrict(int dim, const int64_t *nf, const int64_t *nc, const double *rf,
                        double *rc) {
  const int64_t nzc = nz_cells(dim, nc);
  double scale = 1.0;
  for (int a = 0; a < dim; ++a) scale *= (double)nc[a] / (double)nf[a];
  for (int64_t K = 0; K <= nzc; ++K)
    for (int64_t J = 0; J <= nc[1]; ++J)
      for (int64_t I = 0; I <= nc[0]; ++I) {
        const int64_t pc = vidx(nc, I, J, K);
        if (!is_interior(dim, nc, I, J, K)) {
          rc[pc] = 0.0;
          continue;
        }
        /* every fine vertex whose interpolation uses coarse vertex (I, J, K) */
        double acc = 0.0;
        int64_t klo = 0, khi = 0, jlo, jhi, ilo, ihi;
        if (dim == 3) fine_range(K, nf[2], nc[2], &klo, &khi);
        fine_range(J, nf[1], nc[1], &jlo, &jhi);
        fine_range(I, nf[0], nc[0], &ilo, &ihi);
        for (int64_t k = klo; k <= khi; ++k) {
          const double wz = dim == 3 ? interp_w(k, nf[2], K, nc[2]) : 1.0;
          if (wz == 0.0) continue;
          for (int64_t j = jlo; j <= jhi; ++j) {
            const double wy = interp_w(j, nf[1], J, nc[1]);
            if (wy == 0.0) continue;
            for (int64_t i = ilo; i <= ihi; ++i) {
              const double wx = interp_w(i, nf[0], I, nc[0]);
              if (wx == 0.0) continue;
              acc += wx * wy * wz * rf[vidx(nf, i, j, k)];
            }
          }
        }
        rc[pc] = scale * acc;
      }
}

void oracle_mg_prolong_add(int dim, const int64_t *nf, const int64_t *nc, const double *ec,
                           double *uf) {
  const int64_t nzf = nz_cells(dim, nf), nzc = nz_cells(dim, nc);
  for (int64_t k = 0; k <= nzf; ++k)
    for (int64_t j = 0; j <= nf[1]; ++j)
      for (int64_t i = 0; i <= nf[0]; ++i) {
        if (!is_interior(dim, nf, i, j, k)) continue;
        /* the coarse vertices at or just left of the fine position, and the next */
        double acc = 0.0;
        const int64_t K0 = dim == 3 ? (k * nc[2]) / nf[2] : 0, J0 = (j * nc[1]) / nf[1],
                      I0 = (i * nc[0]) / nf[0];
        const int64_t K1 = dim == 3 && K0 < nzc ? K0 + 1 : K0, J1 = J0 < nc[1] ? J0 + 1 : J0,
                      I1 = I0 < nc[0] ? I0 + 1 : I0;
        for (int64_t K = K0; K <= K1; ++K) {
          const double wz = dim == 3 ? interp_w(k, nf[2], K, nc[2]) : 1.0;
          if (wz == 0.0) continue;
          for (int64_t J = J0; J <= J1; ++J) {
            const double wy = interp_w(j, nf[1], J, nc[1]);
            if (wy == 0.0) continue;
            for (int64_t I = I0; I <= I1; ++I) {
              const double wx = interp_w(i, nf[0], I, nc[0]);
              if (wx == 0.0) continue;
              acc += wx * wy * wz * ec[vidx(nc, I, J, K)];
            }
          }
        }
        uf[vidx(nf, i, j, k)] += acc;
      }
}

static void mg_vcycle(int dim, const int64_t *n, double h, double *u, const double *f,
                      int level, int levels, int pre, int post, int coarse_sweeps) {
  int64_t nc[3];
  if (level == levels - 1 || !mg_coarsen(dim, n, nc)) {
    oracle_gs_coloured(dim, n, h, u, f, coarse_sweeps, 1);
    return;
  }
  const int64_t np = num_points(dim, n);
  const int64_t npc = num_points(dim, nc);
  double *r = (double *)malloc((size_t)np * sizeof(double));
  double *rc = (double *)malloc((size_t)npc * sizeof(double));
  double *ec = (double *)calloc((size_t)npc, sizeof(double));
  double nrm[2];
  oracle_gs_coloured(dim, n, h, u, f, pre, 1);
  oracle_residual(dim, n, h, u, f, r, nrm, 1);
  oracle_mg_restrict(dim, n, nc, r, rc);
  const double hc = h * (double)n[0] / (double)nc[0];
  mg_vcycle(dim, nc, hc, ec, rc, level + 1, levels, pre, post, coarse_sweeps);
  oracle_mg_prolong_add(dim, n, nc, ec, u);
  oracle_gs_coloured(dim, n, h, u, f, post, 1);
  free(r);
  free(rc);
  free(ec);
}

void oracle_mg_vcycle(int dim, const int64_t *n, double h, double *u, const double *f,
                      int levels, int pre, int post, int coarse_sweeps) {
  mg_vcycle(dim, n, h, u, f, 0, levels, pre, post, coarse_sweeps);
}

int oracle_mg_solve(int dim, const int64_t *n, double h, double *u, const double *f,
                    double tol, int max_cycles, int levels, int pre, int post,
                    int coarse_sweeps, double *relres, int *converged) {
  const int64_t np = num_points(dim, n);
  double *r = (double *)malloc((size_t)np * sizeof(double));
  int k = 0;
  *converged = 0;
  for (;;) {
    double nrm[2];
    oracle_residual(dim, n, h, u, f, r, nrm, 1);
    const double rho = nrm[1] > 0.0 ? sqrt(nrm[0]) / sqrt(nrm[1]) : sqrt(nrm[0]);
    if (relres) relres[k] = rho;
    if (rho <= tol) {
      *converged = 1;
      break;
    }
    if (k >= max_cycles) break;
    mg_vcycle(dim, n, h, u, f, 0, levels, pre, post, coarse_sweeps);
    ++k;
  }
  free(r);
  return k;
}

/* --------------------------------------- 5/7-point finite differences, red-black */

/* The compact 2d+1-point stencils of Section 2 (Fig. 1 middle prints the 2D 5-point
 * one: centre 4, face neighbours -1): S u = 2d u - (sum of the 2d face neighbours),
 * A = S / h^2 with the same Dirichlet convention as the Q1 functions.  Section 3 colours
 * these with two colours (red-black); Algorithm 1 indexes the unknowns from 1 and its
 * first pass visits the cells with x + y odd.  With the unknowns at our interior
 * vertices 1..n-1 (x = i, y = j, z = k) the first pass is (i + j + k) odd, the second
 * (i + j + k) even, lexicographic inside a pass. */

double oracle_fd_weight(int dim, int dx, int dy, int dz) {
  const int off = (dx != 0) + (dy != 0) + (dz != 0);
  if (dim == 2 && dz != 0) return 0.0;
  if (off == 0) return 2.0 * dim;
  return off == 1 ? -1.0 : 0.0;
}

static double fd_neighbour_sum(int dim, const int64_t *n, const double *u, int64_t i,
                               int64_t j, int64_t k) {
  /* face neighbours in the order x-, x+, y-, y+, z-, z+ */
  double s = u[vidx(n, i - 1, j, k)] + u[vidx(n, i + 1, j, k)];
  s += u[vidx(n, i, j - 1, k)] + u[vidx(n, i, j + 1, k)];
  if (dim == 3) s += u[vidx(n, i, j, k - 1)] + u[vidx(n, i, j, k + 1)];
  return s;
}

void oracle_fd_apply(int dim, const int64_t *n, double h, const double *u, double *y) {
  const int64_t nzc = nz_cells(dim, n);
  const double h2 = h * h, c = 2.0 * dim;
  for (int64_t k = 0; k <= nzc; ++k)
    for (int64_t j = 0; j <= n[1]; ++j)
      for (int64_t i = 0; i <= n[0]; ++i) {
        const int64_t p = vidx(n, i, j, k);
        y[p] = is_interior(dim, n, i, j, k)
                   ? (c * u[p] - fd_neighbour_sum(dim, n, u, i, j, k)) / h2
                   : 0.0;
      }
}

void oracle_fd_gs_redblack(int dim, const int64_t *n, double h, double *u,
                           const double *f, int sweeps) {
  const int64_t nzc = nz_cells(dim, n);
  const double h2 = h * h, c = 2.0 * dim;
  for (int s = 0; s < sweeps; ++s)
    for (int pass = 0; pass < 2; ++pass) {
      const int64_t parity = pass == 0 ? 1 : 0; /* odd first */
      for (int64_t k = 0; k <= nzc; ++k)
        for (int64_t j = 0; j <= n[1]; ++j)
          for (int64_t i = 0; i <= n[0]; ++i) {
            if (!is_interior(dim, n, i, j, k) || ((i + j + k) & 1) != parity) continue;
            const int64_t p = vidx(n, i, j, k);
            u[p] = (h2 * f[p] + fd_neighbour_sum(dim, n, u, i, j, k)) / c;
          }
    }
}

void oracle_fd_jacobi(int dim, const int64_t *n, double h, double *u, const double *f,
                      double *work, double omega, int sweeps) {
  const int64_t nzc = nz_cells(dim, n), np = num_points(dim, n);
  const double h2 = h * h, c = 2.0 * dim;
  for (int s = 0; s < sweeps; ++s) {
    for (int64_t k = 0; k <= nzc; ++k)
      for (int64_t j = 0; j <= n[1]; ++j)
        for (int64_t i = 0; i <= n[0]; ++i) {
          const int64_t p = vidx(n, i, j, k);
          if (!is_interior(dim, n, i, j, k)) {
            work[p] = u[p];
            continue;
          }
          /* u + omega D^-1 (f - A u), D = 2d / h^2 */
          const double Au = (c * u[p] - fd_neighbour_sum(dim, n, u, i, j, k)) / h2;
          work[p] = u[p] + omega * (h2 / c) * (f[p] - Au);
        }
    memcpy(u, work, (size_t)np * sizeof(double));
  }
}

void oracle_fd_residual(int dim, const int64_t *n, double h, const double *u,
                        const double *f, double *r, double *norms2) {
  const int64_t nzc = nz_cells(dim, n), np = num_points(dim, n);
  double *res = r ? r : (double *)malloc((size_t)np * sizeof(double));
  oracle_fd_apply(dim, n, h, u, res);
  double rr = 0.0, ff = 0.0;
  for (int64_t k = 0; k <= nzc; ++k)
    for (int64_t j = 0; j <= n[1]; ++j)
      for (int64_t i = 0; i <= n[0]; ++i) {
        const int64_t p = vidx(n, i, j, k);
        if (!is_interior(dim, n, i, j, k)) {
          res[p] = 0.0;
          continue;
        }
        res[p] = f[p] - res[p];
        rr += res[p] * res[p];
        ff += f[p] * f[p];
      }
  norms2[0] = rr;
  norms2[1] = ff;
  if (!r) free(res);
}

/* ------------------------------------------- expensive stencil evaluations S(k) */

/* Section 2 parameterises every stencil evaluation S(k) by a cost k, and Section 4
 * realises k > 0 by adding k evaluations of sin to the prescribed entry: k = 100 on
 * every vertex (homogeneous) or k running linearly from 0 to 99 over the mesh
 * (heterogeneous: the first hundredth of the vertices uses the plain stencil, the next
 * adds one sin evaluation, ...).  Our reading, for the red-black finite-difference sweep:
 * the diagonal entry of vertex p becomes 2d + eps * sigma_k(p) / k with
 *   sigma_k(p) = sum_{m=1..k} sin(m * theta_p),  theta_p = idx_p * 2^-20,  eps = 2^-20,
 * idx_p the lexicographic index of p among the interior vertices (x fastest), and
 * k(p) = kmax (uniform) or floor(kmax * idx_p / N) (linear; N interior vertices).  The
 * perturbation is below 2^-20 relative: the operator stays the FD Laplacian to six
 * digits while every update pays for its k sin evaluations. */

static int64_t interior_index(int dim, const int64_t *n, int64_t i, int64_t j, int64_t k) {
  const int64_t rowlen = n[0] - 1, plane = (n[0] - 1) * (n[1] - 1);
  return (dim == 3 ? (k - 1) * plane : 0) + (j - 1) * rowlen + (i - 1);
}

double oracle_cost_diagonal(int dim, const int64_t *n, int mode, int kmax, int64_t i,
                            int64_t j, int64_t k) {
  const int64_t idx = interior_index(dim, n, i, j, k);
  const int64_t N = (n[0] - 1) * (n[1] - 1) * (dim == 3 ? n[2] - 1 : 1);
  int64_t kk = 0;
  if (mode == 1) kk = kmax;
  if (mode == 2) kk = (int64_t)kmax * idx / N;
  double diag = 2.0 * dim;
  if (kk > 0) {
    const double theta = (double)idx * 0x1p-20;
    double sigma = 0.0;
    for (int64_t m = 1; m <= kk; ++m) sigma += sin((double)m * theta);
    diag += 0x1p-20 * (sigma / (double)kk);
  }
  return diag;
}

void oracle_fd_gs_redblack_cost(int dim, const int64_t *n, double h, double *u,
                                const double *f, int sweeps, int mode, int kmax) {
  const int64_t nzc = nz_cells(dim, n);
  const double h2 = h * h;
  for (int s = 0; s < sweeps; ++s)
    for (int pass = 0; pass < 2; ++pass) {
      const int64_t parity = pass == 0 ? 1 : 0;
      for (int64_t k = 0; k <= nzc; ++k)
        for (int64_t j = 0; j <= n[1]; ++j)
          for (int64_t i = 0; i <= n[0]; ++i) {
            if (!is_interior(dim, n, i, j, k) || ((i + j + k) & 1) != parity) continue;
            const int64_t p = vidx(n, i, j, k);
            const double d = oracle_cost_diagonal(dim, n, mode, kmax, i, j, k);
            u[p] = (h2 * f[p] + fd_neighbour_sum(dim, n, u, i, j, k)) / d;
          }
    }
}
