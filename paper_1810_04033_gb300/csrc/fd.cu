// Compact 2d+1-point finite-difference stencils (Section 2; Fig. 1 middle prints the
// 2D 5-point one) with red-black colouring (Section 3): S u = 2d u - (sum of the 2d
// face neighbours), A = S / h^2, Dirichlet data in the boundary vertices.
//
// Red-black Gauss-Seidel runs one in-place pass per colour: a vertex of one colour
// has only neighbours of the other colour, so a pass reads nothing it writes.  The
// first pass updates the interior vertices with (i + j + k) odd, the second the even
// ones (Algorithm 1's order, its 1-based unknowns being our interior vertices).
//
// One CTA per x-row (grid-stride over rows), one thread per vertex of the row; the
// neighbour rows come through L1/L2.  Arithmetic is plain FP64 (a handful of adds per
// update); the sum order is (x- + x+) + (y- + y+) + (z- + z+).  The residual's norms
// use a fixed grid and a fixed-order two-level reduction (the same bits on every call).
#include <cuda_runtime.h>
#include <stdint.h>

#include "cost.cuh"
#include "internal.h"

namespace stencil {
namespace {

constexpr int FD_THREADS = 256;

enum { FD_APPLY = 0, FD_JACOBI = 1, FD_RESIDUAL = 2, FD_GS = 3, FD_GS_COST = 4 };

struct FdArgs {
  Geo q;
  int dim;
  const double *u;
  const double *f;
  double *out;        // y, u_new or r (may be null for the residual); u itself for GS
  double inv_h2;      // 1 / h^2
  double c1;          // Jacobi: omega h^2 / (2d); GS: h^2 / (2d)
  double inv_c;       // GS: 1 / (2d)
  int parity;         // GS: colour of this pass, (i + j + k) & 1
  int cost_mode;      // GS with S(k): COST_UNIFORM or COST_LINEAR (cost.cuh)
  int kmax;
  double h2;          // h^2
  double *partials;   // residual: 2 per CTA
  unsigned *counter;  // residual: CTAs finished
  double *norms2;     // residual: [sum r^2, sum f^2]
};

template <int OP>
__global__ void __launch_bounds__(FD_THREADS) k_fd(FdArgs a) {
  __shared__ double sh[2 * FD_THREADS / 32];
  __shared__ bool last;
  const Geo &q = a.q;
  const int64_t nrows = (q.nz + 1) * (q.ny + 1);
  const double c = 2.0 * a.dim;
  double rr = 0.0, ff = 0.0;
  for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int64_t k = row / (q.ny + 1), j = row % (q.ny + 1);
    const bool row_in = j > 0 && j < q.ny && (a.dim == 2 || (k > 0 && k < q.nz));
    const int64_t base = k * q.plane + j * q.pitch;
    const double *u = a.u + base;
    constexpr bool GS = OP == FD_GS || OP == FD_GS_COST;
    if (GS && !row_in) continue;
    // GS: only the vertices of this pass's colour, every second one of the row
    const int64_t i_first = GS ? 1 + ((a.parity + 1 + j + k) & 1) : 0;
    const int64_t i_step = GS ? 2 : 1;
    for (int64_t i = i_first + i_step * threadIdx.x; i <= q.nx; i += i_step * FD_THREADS) {
      const bool inner = row_in && i > 0 && i < q.nx;
      if (GS) {
        if (!inner) continue;
      } else if (!inner) {
        if (OP == FD_APPLY) a.out[base + i] = 0.0;
        if (OP == FD_JACOBI) a.out[base + i] = u[i];
        if (OP == FD_RESIDUAL && a.out) a.out[base + i] = 0.0;
        continue;
      }
      double s = (u[i - 1] + u[i + 1]) + (u[i - q.pitch] + u[i + q.pitch]);
      if (a.dim == 3) s += u[i - q.plane] + u[i + q.plane];
      if (OP == FD_GS) {
        a.out[base + i] = fma(a.c1, a.f[base + i], s * a.inv_c);
        continue;
      }
      if (OP == FD_GS_COST) {
        const double d = cost_diagonal(q, a.dim, a.cost_mode, a.kmax, i, j, k);
        a.out[base + i] = (a.h2 * a.f[base + i] + s) / d;
        continue;
      }
      const double Au = fma(c, u[i], -s) * a.inv_h2;
      if (OP == FD_APPLY) {
        a.out[base + i] = Au;
      } else if (OP == FD_JACOBI) {
        a.out[base + i] = fma(a.c1, a.f[base + i] - Au, u[i]);
      } else {
        const double fv = a.f[base + i], r = fv - Au;
        if (a.out) a.out[base + i] = r;
        rr = fma(r, r, rr);
        ff = fma(fv, fv, ff);
      }
    }
  }
  if (OP != FD_RESIDUAL) return;
  // fixed-order reduction: warp, CTA, then the last CTA adds the partials in order
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
    ff += __shfl_xor_sync(0xffffffffu, ff, o);
  }
  if (lane == 0) {
    sh[2 * w] = rr;
    sh[2 * w + 1] = ff;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int k = 0; k < FD_THREADS / 32; ++k) {
      s0 += sh[2 * k];
      s1 += sh[2 * k + 1];
    }
    a.partials[2 * blockIdx.x] = s0;
    a.partials[2 * blockIdx.x + 1] = s1;
    __threadfence();
    last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s0 = 0.0, s1 = 0.0;
  for (unsigned k = threadIdx.x; k < gridDim.x; k += FD_THREADS) {
    s0 += __ldcg(a.partials + 2 * k);
    s1 += __ldcg(a.partials + 2 * k + 1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  __syncthreads();
  if (lane == 0) {
    sh[2 * w] = s0;
    sh[2 * w + 1] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int k = 0; k < FD_THREADS / 32; ++k) {
      t0 += sh[2 * k];
      t1 += sh[2 * k + 1];
    }
    a.norms2[0] = t0;
    a.norms2[1] = t1;
    *a.counter = 0u;
  }
}

unsigned fd_blocks(const Geo &q) {
  const int64_t rows = (q.nz + 1) * (q.ny + 1);
  const int64_t cap = 8ll * device_sm_count();
  return (unsigned)(rows < cap ? rows : cap);
}

FdArgs fd_args(const Geo &q, int dim) {
  FdArgs a{};
  a.q = q;
  a.dim = dim;
  a.inv_h2 = 1.0 / (q.h * q.h);
  return a;
}

}  // namespace

size_t fd_reduce_bytes(const Geo &q) { return 16 + (size_t)fd_blocks(q) * 2 * sizeof(double); }

cudaError_t launch_fd_apply(const Geo &q, int dim, const double *u, double *y, cudaStream_t s) {
  FdArgs a = fd_args(q, dim);
  a.u = u;
  a.out = y;
  k_fd<FD_APPLY><<<fd_blocks(q), FD_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fd_jacobi(const Geo &q, int dim, const double *u, const double *f, double *unew, double omega,
                             cudaStream_t s) {
  FdArgs a = fd_args(q, dim);
  a.u = u;
  a.f = f;
  a.out = unew;
  a.c1 = omega * q.h * q.h / (2.0 * dim);
  k_fd<FD_JACOBI><<<fd_blocks(q), FD_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fd_residual(const Geo &q, int dim, const double *u, const double *f, double *r, double *norms2,
                               void *scratch, cudaStream_t s) {
  FdArgs a = fd_args(q, dim);
  a.u = u;
  a.f = f;
  a.out = r;
  a.counter = (unsigned *)scratch;  // counter first, partials after (same layout everywhere)
  a.partials = (double *)((char *)scratch + 16);
  a.norms2 = norms2;
  k_fd<FD_RESIDUAL><<<fd_blocks(q), FD_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fd_gs_redblack(const Geo &q, int dim, double *u, const double *f, int sweeps, cudaStream_t s) {
  FdArgs a = fd_args(q, dim);
  a.u = u;
  a.f = f;
  a.out = u;
  a.c1 = q.h * q.h / (2.0 * dim);
  a.inv_c = 1.0 / (2.0 * dim);
  for (int it = 0; it < sweeps; ++it)
    for (int pass = 0; pass < 2; ++pass) {
      a.parity = pass == 0 ? 1 : 0;
      k_fd<FD_GS><<<fd_blocks(q), FD_THREADS, 0, s>>>(a);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

cudaError_t launch_fd_gs_redblack_cost(const Geo &q, int dim, double *u, const double *f, int sweeps, int mode,
                                       int kmax, cudaStream_t s) {
  FdArgs a = fd_args(q, dim);
  a.u = u;
  a.f = f;
  a.out = u;
  a.h2 = q.h * q.h;
  a.cost_mode = mode;
  a.kmax = kmax;
  for (int it = 0; it < sweeps; ++it)
    for (int pass = 0; pass < 2; ++pass) {
      a.parity = pass == 0 ? 1 : 0;
      k_fd<FD_GS_COST><<<fd_blocks(q), FD_THREADS, 0, s>>>(a);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

}  // namespace stencil
