// Geometric multigrid V-cycle around the coloured Gauss-Seidel sweeps (Section 1: the
// paper's sweeps are the smoothers of matrix-free multigrid codes).
//
// Hierarchy (vertex-centred): the coarse grid has n/2 cells per axis when every n is
// even (every second vertex), or ceil(n/2) on every axis when all n are equal (then the
// coarse vertices are not fine vertices); coarse cells are cubes of side h n / n_c.
// Grids are coarsened while every n >= 4.
// Transfers, with fine vertex i at position i / n_f and coarse vertex I at I / n_c (in
// units of the domain side) and the 1D weight w(i, I) = 1 - |i n_c - I n_f| / n_f
// where positive:
//   prolongation P: d-linear interpolation (weights w per axis), added to the fine
//     interior (the coarse correction's boundary is 0);
//   restriction R = (n_c / n_f)^d P^T (full weighting for nested grids), so that
//     R A_h P = A_2h for the Q1 operator A = S / h^2 on nested grids.
// V-cycle on level l: `pre` sweeps; r = f - A u (FP64); f_{l+1} = R r; e_{l+1} = 0;
// V-cycle on level l + 1 (on the coarsest level: `coarse_sweeps` sweeps); u += P e;
// `post` sweeps.  All launches are stream-ordered; the solve reads one norm pair per
// cycle back to the host.
//
// Both transfer kernels are one thread per output vertex (x fastest, grid-stride over
// rows); the fine values a coarse vertex gathers (3 per axis nested, up to 4 otherwise)
// and the coarse values a fine vertex interpolates (up to 2 per axis) come from L1/L2.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

#include "internal.h"

namespace stencil {
namespace {

constexpr int MG_THREADS = 256;

// 1D interpolation weight of coarse vertex I (nc cells) at fine vertex i (nf cells):
// 1 - |i nc - I nf| / nf where positive (inv_nf = 1 / nf).
__device__ __forceinline__ double interp_w(int64_t i, int64_t nf, int64_t I, int64_t nc, double inv_nf) {
  int64_t d = i * nc - I * nf;
  d = d < 0 ? -d : d;
  return d >= nf ? 0.0 : (double)(nf - d) * inv_nf;
}

// Fine indices that see coarse vertex I: |i nc - I nf| < nf.
__device__ __forceinline__ void fine_range(int64_t I, int64_t nf, int64_t nc, int64_t &lo, int64_t &hi) {
  lo = ((I - 1) * nf) / nc + 1;  // I >= 1: floor division of a non-negative value
  hi = ((I + 1) * nf + nc - 1) / nc - 1;
  if (lo < 0) lo = 0;
  if (hi > nf) hi = nf;
}

struct Dims {
  int64_t f[3], c[3];  // cells per axis (z entry 0 in 2D)
  double inv_f[3];     // 1 / f (1 for an unused axis)
};


// rc = R rf on the interior of the coarse grid, 0 on its boundary.  NESTED: n_f = 2 n_c
// on every axis (weights 1 and 1/2 at fine offsets 0 and +-1 around 2I, grouped).
template <bool NESTED>
__global__ void __launch_bounds__(MG_THREADS) k_mg_restrict(Geo qf, Geo qc, Dims d, int dim, double scale,
                                                           const double *__restrict__ rf, double *__restrict__ rc) {
  const int64_t nrows = (qc.nz + 1) * (qc.ny + 1);
  for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int64_t K = row / (qc.ny + 1), J = row % (qc.ny + 1);
    const bool row_in = J > 0 && J < qc.ny && (dim == 2 || (K > 0 && K < qc.nz));
    double *out = rc + K * qc.plane + J * qc.pitch;
    int64_t klo = 0, khi = 0, jlo = 0, jhi = 0;
    if (row_in && !NESTED) {
      if (dim == 3) fine_range(K, d.f[2], d.c[2], klo, khi);
      fine_range(J, d.f[1], d.c[1], jlo, jhi);
    }
    for (int64_t I = threadIdx.x; I <= qc.nx; I += MG_THREADS) {
      if (!row_in || I == 0 || I == qc.nx) {
        out[I] = 0.0;
        continue;
      }
      double acc = 0.0;
      if (NESTED) {
        // grouped by weight: centre 1, faces 1/2, edges 1/4, corners 1/8 (3D); the
        // 1/2^d scale is applied by the caller's `scale`
        const double *p = rf + (dim == 3 ? 2 * K * qf.plane : 0) + 2 * J * qf.pitch + 2 * I;
        const int64_t sy = qf.pitch, sz = qf.plane;
        const double c = p[0];
        double fa = (p[-1] + p[1]) + (p[-sy] + p[sy]);
        double ed = (p[-sy - 1] + p[-sy + 1]) + (p[sy - 1] + p[sy + 1]);
        double co = 0.0;
        if (dim == 3) {
          fa += p[-sz] + p[sz];
          ed += ((p[-sz - 1] + p[-sz + 1]) + (p[-sz - sy] + p[-sz + sy])) +
                ((p[sz - 1] + p[sz + 1]) + (p[sz - sy] + p[sz + sy]));
          co = ((p[-sz - sy - 1] + p[-sz - sy + 1]) + (p[-sz + sy - 1] + p[-sz + sy + 1])) +
               ((p[sz - sy - 1] + p[sz - sy + 1]) + (p[sz + sy - 1] + p[sz + sy + 1]));
          acc = c + 0.5 * fa + 0.25 * ed + 0.125 * co;
        } else {
          acc = c + 0.5 * fa + 0.25 * ed;
        }
      } else {
        int64_t ilo, ihi;
        fine_range(I, d.f[0], d.c[0], ilo, ihi);
        for (int64_t k = klo; k <= khi; ++k) {
          const double wz = dim == 3 ? interp_w(k, d.f[2], K, d.c[2], d.inv_f[2]) : 1.0;
          for (int64_t j = jlo; j <= jhi; ++j) {
            const double wyz = interp_w(j, d.f[1], J, d.c[1], d.inv_f[1]) * wz;
            const double *p = rf + k * qf.plane + j * qf.pitch;
            for (int64_t i = ilo; i <= ihi; ++i) acc += interp_w(i, d.f[0], I, d.c[0], d.inv_f[0]) * wyz * p[i];
          }
        }
      }
      out[I] = scale * acc;
    }
  }
}

// uf += P ec on the interior of the fine grid.
template <bool NESTED>
__global__ void __launch_bounds__(MG_THREADS) k_mg_prolong_add(Geo qf, Geo qc, Dims d, int dim,
                                                              const double *__restrict__ ec,
                                                              double *__restrict__ uf) {
  const int64_t nrows = (qf.nz + 1) * (qf.ny + 1);
  for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int64_t k = row / (qf.ny + 1), j = row % (qf.ny + 1);
    if (j == 0 || j == qf.ny || (dim == 3 && (k == 0 || k == qf.nz))) continue;
    const int64_t K0 = dim == 3 ? (NESTED ? k >> 1 : (k * d.c[2]) / d.f[2]) : 0;
    const int64_t J0 = NESTED ? j >> 1 : (j * d.c[1]) / d.f[1];
    const int64_t K1 = dim == 3 && K0 < d.c[2] ? K0 + 1 : K0, J1 = J0 < d.c[1] ? J0 + 1 : J0;
    double *out = uf + k * qf.plane + j * qf.pitch;
    for (int64_t i = 1 + threadIdx.x; i < qf.nx; i += MG_THREADS) {
      const int64_t I0 = NESTED ? i >> 1 : (i * d.c[0]) / d.f[0], I1 = I0 < d.c[0] ? I0 + 1 : I0;
      double acc = 0.0;
      if (NESTED) {
        // sum of the 1, 2, 4 or 8 coarse values around the fine vertex, times 2^-(odd axes)
        const bool ox = i & 1, oy = j & 1, oz = dim == 3 && (k & 1);
        const double *pc = ec + K0 * qc.plane + J0 * qc.pitch + I0;
        double sum = ox ? pc[0] + pc[1] : pc[0];
        if (oy) sum += ox ? pc[qc.pitch] + pc[qc.pitch + 1] : pc[qc.pitch];
        if (oz) {
          const double *pz = pc + qc.plane;
          double s2 = ox ? pz[0] + pz[1] : pz[0];
          if (oy) s2 += ox ? pz[qc.pitch] + pz[qc.pitch + 1] : pz[qc.pitch];
          sum += s2;
        }
        const int m = (int)ox + (int)oy + (int)oz;
        acc = m == 0 ? sum : sum * (m == 1 ? 0.5 : (m == 2 ? 0.25 : 0.125));
      } else {
        for (int64_t K = K0; K <= K1; ++K) {
          const double wz = dim == 3 ? interp_w(k, d.f[2], K, d.c[2], d.inv_f[2]) : 1.0;
          if (wz == 0.0) continue;
          for (int64_t J = J0; J <= J1; ++J) {
            const double wyz = interp_w(j, d.f[1], J, d.c[1], d.inv_f[1]) * wz;
            if (wyz == 0.0) continue;
            const double *pc = ec + K * qc.plane + J * qc.pitch;
            for (int64_t I = I0; I <= I1; ++I) {
              const double w = interp_w(i, d.f[0], I, d.c[0], d.inv_f[0]) * wyz;
              if (w != 0.0) acc += w * pc[I];
            }
          }
        }
      }
      out[i] += acc;
    }
  }
}

unsigned mg_blocks(const Geo &q) {
  const int64_t rows = (q.nz + 1) * (q.ny + 1);
  const int64_t cap = 16ll * device_sm_count();
  return (unsigned)(rows < cap ? rows : cap);
}

}  // namespace

bool mg_coarse(const Geo &qf, int dim, Geo &qc) {
  const int64_t n[3] = {qf.nx, qf.ny, dim == 3 ? qf.nz : qf.nx};
  bool all_even = true, all_equal = true;
  for (int a = 0; a < dim; ++a) {
    if (n[a] < 4) return false;
    if (n[a] % 2) all_even = false;
    if (n[a] != n[0]) all_equal = false;
  }
  if (!all_even && !all_equal) return false;
  qc.nx = (qf.nx + 1) / 2;
  qc.ny = (qf.ny + 1) / 2;
  qc.nz = dim == 3 ? (qf.nz + 1) / 2 : 0;
  qc.pitch = qc.nx + 1;
  qc.plane = qc.pitch * (qc.ny + 1);
  qc.h = qf.h * (double)qf.nx / (double)qc.nx;
  return true;
}

int mg_levels(const Geo &q, int dim, int max_levels) {
  Geo g = q, c;
  int L = 1;
  while (L < max_levels && mg_coarse(g, dim, c)) {
    g = c;
    ++L;
  }
  return L;
}

static Dims dims_of(const Geo &qf, const Geo &qc) {
  Dims d;
  d.f[0] = qf.nx, d.f[1] = qf.ny, d.f[2] = qf.nz;
  d.c[0] = qc.nx, d.c[1] = qc.ny, d.c[2] = qc.nz;
  for (int a = 0; a < 3; ++a) d.inv_f[a] = d.f[a] ? 1.0 / (double)d.f[a] : 1.0;
  return d;
}

static bool nested(const Geo &qf, const Geo &qc, int dim) {
  return qf.nx == 2 * qc.nx && qf.ny == 2 * qc.ny && (dim == 2 || qf.nz == 2 * qc.nz);
}

cudaError_t launch_mg_restrict(const Geo &qf, const Geo &qc, int dim, const double *rf, double *rc, cudaStream_t s) {
  double scale = (double)qc.nx / (double)qf.nx * ((double)qc.ny / (double)qf.ny);
  if (dim == 3) scale *= (double)qc.nz / (double)qf.nz;
  if (nested(qf, qc, dim))
    k_mg_restrict<true><<<mg_blocks(qc), MG_THREADS, 0, s>>>(qf, qc, dims_of(qf, qc), dim, scale, rf, rc);
  else
    k_mg_restrict<false><<<mg_blocks(qc), MG_THREADS, 0, s>>>(qf, qc, dims_of(qf, qc), dim, scale, rf, rc);
  return cudaGetLastError();
}

cudaError_t launch_mg_prolong_add(const Geo &qf, const Geo &qc, int dim, const double *ec, double *uf,
                                  cudaStream_t s) {
  if (nested(qf, qc, dim))
    k_mg_prolong_add<true><<<mg_blocks(qf), MG_THREADS, 0, s>>>(qf, qc, dims_of(qf, qc), dim, ec, uf);
  else
    k_mg_prolong_add<false><<<mg_blocks(qf), MG_THREADS, 0, s>>>(qf, qc, dims_of(qf, qc), dim, ec, uf);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ V-cycle driver

static size_t span_bytes_256(const Geo &q) { return ((size_t)span_elems(q) * sizeof(double) + 255) / 256 * 256; }

size_t mg_work_bytes(const Geo &q0, int dim, int levels) {
  // coarse u and f of levels 1..L-1, fine residual of levels 0..L-2
  size_t b = 0;
  Geo q = q0, c;
  for (int l = 0; l < levels; ++l) {
    if (l > 0) b += 2 * span_bytes_256(q);
    if (l < levels - 1) b += span_bytes_256(q);
    if (!mg_coarse(q, dim, c)) break;
    q = c;
  }
  return b;
}

size_t mg_reduce_bytes(const Geo &q0, int dim, int levels) {
  size_t b = 0;
  Geo q = q0, c;
  for (int l = 0; l < levels; ++l) {
    const size_t x = dim == 3 ? ops_fx_reduce_bytes(q) : ops2_reduce_bytes(q);
    b = x > b ? x : b;
    if (!mg_coarse(q, dim, c)) break;
    q = c;
  }
  return b;
}

cudaError_t MgCycle::run(double *u0, const double *f0) {
  return level(0, u0, f0);
}

cudaError_t MgCycle::level(int l, double *u, const double *f) {
  const Geo &q = q_[l];
  cudaError_t e;
  if (l == levels_ - 1) return smooth(q, u, f, coarse_sweeps_);
  if ((e = smooth(q, u, f, pre_))) return e;
  e = dim_ == 3 ? launch_residual_fx3(q, u, f, r_[l], norms_, red_, s_)
                : launch_residual_fx2(q, u, f, r_[l], norms_, red_, s_);
  if (e) return e;
  const Geo &qc = q_[l + 1];
  if ((e = launch_mg_restrict(q, qc, dim_, r_[l], f_[l + 1], s_))) return e;
  if ((e = cudaMemsetAsync(u_[l + 1], 0, (size_t)span_elems(qc) * sizeof(double), s_))) return e;
  if ((e = level(l + 1, u_[l + 1], f_[l + 1]))) return e;
  if ((e = launch_mg_prolong_add(q, qc, dim_, u_[l + 1], u, s_))) return e;
  return smooth(q, u, f, post_);
}

cudaError_t MgCycle::smooth(const Geo &q, double *u, const double *f, int sweeps) {
  if (sweeps <= 0) return cudaSuccess;
  return dim_ == 3 ? launch_gs_sweeps_fx3(q, u, f, sweeps, gs_work_, gs_bounds_, s_)
                   : launch_gs_sweeps_fx2(q, u, f, sweeps, gs_work_, gs_bounds_, s_);
}

bool MgCycle::setup(const Geo &q0, int dim, int levels, int pre, int post, int coarse_sweeps, void *work,
                    double *gs_work, void *gs_bounds, double *norms, void *red, cudaStream_t s) {
  if (levels < 1 || levels > kMaxLevels) return false;
  dim_ = dim;
  levels_ = levels;
  pre_ = pre;
  post_ = post;
  coarse_sweeps_ = coarse_sweeps;
  gs_work_ = gs_work;
  gs_bounds_ = gs_bounds;
  norms_ = norms;
  red_ = red;
  s_ = s;
  char *p = (char *)work;
  q_[0] = q0;
  for (int l = 0; l < levels; ++l) {
    if (l > 0 && !mg_coarse(q_[l - 1], dim, q_[l])) return false;
    const size_t span = span_bytes_256(q_[l]);
    u_[l] = f_[l] = r_[l] = nullptr;
    if (l > 0) {
      u_[l] = (double *)p;
      p += span;
      f_[l] = (double *)p;
      p += span;
    }
    if (l < levels - 1) {
      r_[l] = (double *)p;
      p += span;
    }
  }
  return true;
}

}  // namespace stencil
