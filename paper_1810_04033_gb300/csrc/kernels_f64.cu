// Native FP64 kernels: assembled-stencil apply, element-wise apply with 2^d-colour
// scatter, coloured Gauss-Seidel phases, damped Jacobi and the residual with a
// fixed-order norm reduction.
//
// Operator (Section 2, Fig. 1): A = S/h^2 with the assembled Q1 stencil S.
//   3D: S u = 8/3 u - E/6 - C/12, E = sum of the 12 edge neighbours (two indices
//       differ), C = sum of the 8 corner neighbours; face neighbours have weight 0.
//   2D: S u = 8/3 u - N/3, N = sum of the 8 neighbours.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace stencil {
namespace {

__device__ __forceinline__ int64_t at(const Geo &q, int64_t i, int64_t j, int64_t k) {
  return k * q.plane + j * q.pitch + i;
}

// Edge and corner sums around the vertex at c (3D).
__device__ __forceinline__ void edge_corner_sums(const double *__restrict__ c, int64_t P,
                                                 int64_t Z, double &E, double &C) {
  E = ((c[-1 - P] + c[1 - P]) + (c[-1 + P] + c[1 + P])) +
      ((c[-1 - Z] + c[1 - Z]) + (c[-1 + Z] + c[1 + Z])) +
      ((c[-P - Z] + c[P - Z]) + (c[-P + Z] + c[P + Z]));
  C = ((c[-1 - P - Z] + c[1 - P - Z]) + (c[-1 + P - Z] + c[1 + P - Z])) +
      ((c[-1 - P + Z] + c[1 - P + Z]) + (c[-1 + P + Z] + c[1 + P + Z]));
}

// Sum of the 8 neighbours around c (2D).
__device__ __forceinline__ double ring_sum(const double *__restrict__ c, int64_t P) {
  return ((c[-1 - P] + c[-P]) + (c[1 - P] + c[-1])) + ((c[1] + c[-1 + P]) + (c[P] + c[1 + P]));
}

// ----------------------------------------------------------------- stencil apply

__global__ void k_apply_stencil3(Geo q, const double *__restrict__ u, double *__restrict__ y,
                                 double inv12h2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > q.nx) return;
  for (int64_t k = blockIdx.z; k <= q.nz; k += gridDim.z)
    for (int64_t j = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; j <= q.ny;
         j += (int64_t)gridDim.y * blockDim.y) {
      const int64_t p = at(q, i, j, k);
      if (i == 0 || i == q.nx || j == 0 || j == q.ny || k == 0 || k == q.nz) {
        y[p] = 0.0;
        continue;
      }
      double E, C;
      edge_corner_sums(u + p, q.pitch, q.plane, E, C);
      // S u * 12 = 32 u - 2E - C
      y[p] = fma(32.0, u[p], -fma(2.0, E, C)) * inv12h2;
    }
}

__global__ void k_apply_stencil2(Geo q, const double *__restrict__ u, double *__restrict__ y,
                                 double inv3h2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > q.nx) return;
  for (int64_t j = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; j <= q.ny;
       j += (int64_t)gridDim.y * blockDim.y) {
    const int64_t p = j * q.pitch + i;
    if (i == 0 || i == q.nx || j == 0 || j == q.ny) {
      y[p] = 0.0;
      continue;
    }
    // S u * 3 = 8 u - N
    y[p] = fma(8.0, u[p], -ring_sum(u + p, q.pitch)) * inv3h2;
  }
}

// ------------------------------------------------------------ element-wise apply
// A CTA owns a TX x TY x TZ block of vertices.  It stages u on the block plus a
// one-vertex halo in shared memory, then visits the cells touching its vertices in 2^d
// colour passes; a cell adds K_e u_e into the shared accumulator of its 2^d vertices.
// Cells of one colour share no vertex, so a pass needs no atomics; passes are
// separated by a barrier.  Cells on the tile rim are recomputed by the neighbouring
// CTA as well; each CTA writes only the vertices it owns.
constexpr int EW_TX = 32, EW_TY = 4, EW_TZ = 4;

__global__ void __launch_bounds__(256) k_apply_elementwise3(Geo q, const double *__restrict__ u,
                                                            double *__restrict__ y, double scale) {
  constexpr int SX = EW_TX + 2, SY = EW_TY + 2, SZ = EW_TZ + 2;
  __shared__ double us[SZ][SY][SX];
  __shared__ double ys[SZ][SY][SX];
  const int tid = threadIdx.x;
  const int64_t x0 = (int64_t)blockIdx.x * EW_TX, y0 = (int64_t)blockIdx.y * EW_TY,
                z0 = (int64_t)blockIdx.z * EW_TZ;
  for (int t = tid; t < SX * SY * SZ; t += blockDim.x) {
    const int lx = t % SX, ly = (t / SX) % SY, lz = t / (SX * SY);
    const int64_t gx = x0 - 1 + lx, gy = y0 - 1 + ly, gz = z0 - 1 + lz;
    double v = 0.0;
    if (gx >= 0 && gx <= q.nx && gy >= 0 && gy <= q.ny && gz >= 0 && gz <= q.nz)
      v = u[at(q, gx, gy, gz)];
    us[lz][ly][lx] = v;
    ys[lz][ly][lx] = 0.0;
  }
  __syncthreads();
  // local cells (cx,cy,cz) in [0,SX-1) x [0,SY-1) x [0,SZ-1): global cell x0-1+cx ...
  constexpr int CX = SX - 1, CY = SY - 1, CZ = SZ - 1;
  for (int colour = 0; colour < 8; ++colour) {
    for (int t = tid; t < CX * CY * CZ; t += blockDim.x) {
      const int cx = t % CX, cy = (t / CX) % CY, cz = t / (CX * CY);
      const int64_t gx = x0 - 1 + cx, gy = y0 - 1 + cy, gz = z0 - 1 + cz;
      if (gx < 0 || gx >= q.nx || gy < 0 || gy >= q.ny || gz < 0 || gz >= q.nz) continue;
      if ((int)((gx & 1) + 2 * (gy & 1) + 4 * (gz & 1)) != colour) continue;
      double v[8];
#pragma unroll
      for (int w = 0; w < 8; ++w) v[w] = us[cz + (w >> 2)][cy + ((w >> 1) & 1)][cx + (w & 1)];
      const double T = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        // 12 (K_hat u_e)_w = 5 u_w + (sum of the 3 face-adjacent vertices) - T
        const double F = (v[w ^ 1] + v[w ^ 2]) + v[w ^ 4];
        ys[cz + (w >> 2)][cy + ((w >> 1) & 1)][cx + (w & 1)] += fma(5.0, v[w], F - T);
      }
    }
    __syncthreads();
  }
  for (int t = tid; t < EW_TX * EW_TY * EW_TZ; t += blockDim.x) {
    const int lx = 1 + t % EW_TX, ly = 1 + (t / EW_TX) % EW_TY, lz = 1 + t / (EW_TX * EW_TY);
    const int64_t gx = x0 - 1 + lx, gy = y0 - 1 + ly, gz = z0 - 1 + lz;
    if (gx > q.nx || gy > q.ny || gz > q.nz) continue;
    const bool interior = gx > 0 && gx < q.nx && gy > 0 && gy < q.ny && gz > 0 && gz < q.nz;
    y[at(q, gx, gy, gz)] = interior ? ys[lz][ly][lx] * scale : 0.0;
  }
}

constexpr int EW2_TX = 32, EW2_TY = 8;

__global__ void __launch_bounds__(256) k_apply_elementwise2(Geo q, const double *__restrict__ u,
                                                            double *__restrict__ y, double scale) {
  constexpr int SX = EW2_TX + 2, SY = EW2_TY + 2;
  __shared__ double us[SY][SX];
  __shared__ double ys[SY][SX];
  const int tid = threadIdx.x;
  const int64_t x0 = (int64_t)blockIdx.x * EW2_TX, y0 = (int64_t)blockIdx.y * EW2_TY;
  for (int t = tid; t < SX * SY; t += blockDim.x) {
    const int lx = t % SX, ly = t / SX;
    const int64_t gx = x0 - 1 + lx, gy = y0 - 1 + ly;
    double v = 0.0;
    if (gx >= 0 && gx <= q.nx && gy >= 0 && gy <= q.ny) v = u[gy * q.pitch + gx];
    us[ly][lx] = v;
    ys[ly][lx] = 0.0;
  }
  __syncthreads();
  constexpr int CX = SX - 1, CY = SY - 1;
  for (int colour = 0; colour < 4; ++colour) {
    for (int t = tid; t < CX * CY; t += blockDim.x) {
      const int cx = t % CX, cy = t / CX;
      const int64_t gx = x0 - 1 + cx, gy = y0 - 1 + cy;
      if (gx < 0 || gx >= q.nx || gy < 0 || gy >= q.ny) continue;
      if ((int)((gx & 1) + 2 * (gy & 1)) != colour) continue;
      double v[4];
#pragma unroll
      for (int w = 0; w < 4; ++w) v[w] = us[cy + (w >> 1)][cx + (w & 1)];
      const double T = (v[0] + v[1]) + (v[2] + v[3]);
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        // 6 (K_hat u_e)_w = 6 u_w + (sum of the 2 face-adjacent vertices) - 2 T
        const double F = v[w ^ 1] + v[w ^ 2];
        ys[cy + (w >> 1)][cx + (w & 1)] += fma(6.0, v[w], fma(-2.0, T, F));
      }
    }
    __syncthreads();
  }
  for (int t = tid; t < EW2_TX * EW2_TY; t += blockDim.x) {
    const int lx = 1 + t % EW2_TX, ly = 1 + t / EW2_TX;
    const int64_t gx = x0 - 1 + lx, gy = y0 - 1 + ly;
    if (gx > q.nx || gy > q.ny) continue;
    const bool interior = gx > 0 && gx < q.nx && gy > 0 && gy < q.ny;
    y[gy * q.pitch + gx] = interior ? ys[ly][lx] * scale : 0.0;
  }
}

// ------------------------------------------------------------------ Gauss-Seidel
// 3D: the face weight of S is 0, so vertices whose indices differ only in the x
// parity are not coupled; colours 2m and 2m+1 can therefore be updated in one phase
// with bit-identical results.  A sweep is 4 phases over rows (j&1, k&1) =
// (0,0), (1,0), (0,1), (1,1), i.e. colour pairs {0,1}, {2,3}, {4,5}, {6,7}.
// Update: u_i = 3/8 (h^2 f_i + E/6 + C/12) = 3/8 h^2 f_i + (2E + C)/32.
__global__ void k_gs_phase3(Geo q, double *__restrict__ u, const double *__restrict__ f,
                            int py, int pz, double g) {
  const int64_t i = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= q.nx) return;
  for (int64_t k = 1 + pz + 2 * (int64_t)blockIdx.z; k < q.nz; k += 2 * (int64_t)gridDim.z)
    for (int64_t j = 1 + py + 2 * ((int64_t)blockIdx.y * blockDim.y + threadIdx.y); j < q.ny;
         j += 2 * (int64_t)gridDim.y * blockDim.y) {
      // py, pz are the offsets from 1 of the first row / plane of this phase
      const int64_t p = at(q, i, j, k);
      double E, C;
      edge_corner_sums(u + p, q.pitch, q.plane, E, C);
      u[p] = fma(fma(2.0, E, C), 0.03125, g * f[p]);
    }
}

// 2D: every colour (px, py) is its own phase; u_i = 3/8 h^2 f_i + N/8.
__global__ void k_gs_colour2(Geo q, double *__restrict__ u, const double *__restrict__ f,
                             int px, int py, double g) {
  const int64_t i = 1 + px + 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= q.nx) return;
  for (int64_t j = 1 + py + 2 * ((int64_t)blockIdx.y * blockDim.y + threadIdx.y); j < q.ny;
       j += 2 * (int64_t)gridDim.y * blockDim.y) {
    const int64_t p = j * q.pitch + i;
    u[p] = fma(ring_sum(u + p, q.pitch), 0.125, g * f[p]);
  }
}

// ------------------------------------------------------------------------ Jacobi
__global__ void k_jacobi3(Geo q, const double *__restrict__ u, const double *__restrict__ f,
                          double *__restrict__ un, double h2, double w38) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > q.nx) return;
  for (int64_t k = blockIdx.z; k <= q.nz; k += gridDim.z)
    for (int64_t j = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; j <= q.ny;
         j += (int64_t)gridDim.y * blockDim.y) {
      const int64_t p = at(q, i, j, k);
      if (i == 0 || i == q.nx || j == 0 || j == q.ny || k == 0 || k == q.nz) {
        un[p] = u[p];
        continue;
      }
      double E, C;
      edge_corner_sums(u + p, q.pitch, q.plane, E, C);
      const double Su = fma(32.0, u[p], -fma(2.0, E, C)) * (1.0 / 12.0);
      un[p] = fma(w38, fma(h2, f[p], -Su), u[p]);
    }
}

__global__ void k_jacobi2(Geo q, const double *__restrict__ u, const double *__restrict__ f,
                          double *__restrict__ un, double h2, double w38) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > q.nx) return;
  for (int64_t j = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; j <= q.ny;
       j += (int64_t)gridDim.y * blockDim.y) {
    const int64_t p = j * q.pitch + i;
    if (i == 0 || i == q.nx || j == 0 || j == q.ny) {
      un[p] = u[p];
      continue;
    }
    const double Su = fma(8.0, u[p], -ring_sum(u + p, q.pitch)) * (1.0 / 3.0);
    un[p] = fma(w38, fma(h2, f[p], -Su), u[p]);
  }
}

// ---------------------------------------------------------------------- residual
// Rows (all (k, j) pairs) are dealt round-robin to kReduceBlocks CTAs; each thread
// strides over x.  Per-thread partial sums, a fixed butterfly inside the CTA, one
// partial per CTA, and the last CTA to finish adds the partials in index order.  The
// summation order depends only on the grid and the fixed CTA count, so repeated calls
// return identical bits.
constexpr int RED_THREADS = 256;

__device__ __forceinline__ void block_sum2(double &a, double &b, double *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sh[2 * w] = a;
    sh[2 * w + 1] = b;
  }
  __syncthreads();
  if (w == 0) {
    constexpr int NW = RED_THREADS / 32;
    a = l < NW ? sh[2 * l] : 0.0;
    b = l < NW ? sh[2 * l + 1] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
  }
}

__global__ void __launch_bounds__(RED_THREADS) k_residual(Geo q, int dim, const double *__restrict__ u,
                                                          const double *__restrict__ f,
                                                          double *__restrict__ r, double *norms2,
                                                          double *partials, unsigned *counter,
                                                          double inv_h2) {
  __shared__ double sh[2 * RED_THREADS / 32];
  __shared__ bool last;
  double rr = 0.0, ff = 0.0;
  const int64_t nrows = (q.nz + 1) * (q.ny + 1);
  for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int64_t k = row / (q.ny + 1), j = row % (q.ny + 1);
    const bool row_inner = j > 0 && j < q.ny && (dim == 2 || (k > 0 && k < q.nz));
    for (int64_t i = threadIdx.x; i <= q.nx; i += blockDim.x) {
      const int64_t p = at(q, i, j, k);
      if (!row_inner || i == 0 || i == q.nx) {
        if (r) r[p] = 0.0;
        continue;
      }
      double Su;
      if (dim == 3) {
        double E, C;
        edge_corner_sums(u + p, q.pitch, q.plane, E, C);
        Su = fma(32.0, u[p], -fma(2.0, E, C)) * (1.0 / 12.0);
      } else {
        Su = fma(8.0, u[p], -ring_sum(u + p, q.pitch)) * (1.0 / 3.0);
      }
      const double fp = f[p];
      const double rp = fma(-Su, inv_h2, fp);
      if (r) r[p] = rp;
      rr = fma(rp, rp, rr);
      ff = fma(fp, fp, ff);
    }
  }
  block_sum2(rr, ff, sh);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = rr;
    partials[2 * blockIdx.x + 1] = ff;
    __threadfence();
    const unsigned ticket = atomicAdd(counter, 1u);
    last = ticket == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double a = 0.0, b = 0.0;
  for (int t = threadIdx.x; t < (int)gridDim.x; t += blockDim.x) {
    a += __ldcg(partials + 2 * t);
    b += __ldcg(partials + 2 * t + 1);
  }
  __syncthreads();  // sh reuse
  block_sum2(a, b, sh);
  if (threadIdx.x == 0) {
    norms2[0] = a;
    norms2[1] = b;
    *counter = 0u;  // ready for the next call on this scratch
  }
}

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }
inline unsigned clamp_grid(int64_t v, unsigned lim) {
  return v < 1 ? 1u : (v > lim ? lim : (unsigned)v);
}

}  // namespace

cudaError_t launch_apply_stencil_f64(const Geo &q, int dim, const double *u, double *y,
                                     cudaStream_t s) {
  const double h2 = q.h * q.h;
  if (dim == 3) {
    dim3 b(128, 2), gr(cdiv(q.nx + 1, 128), clamp_grid(cdiv(q.ny + 1, 2), 65535),
                       clamp_grid(q.nz + 1, 65535));
    k_apply_stencil3<<<gr, b, 0, s>>>(q, u, y, 1.0 / (12.0 * h2));
  } else {
    dim3 b(128, 2), gr(cdiv(q.nx + 1, 128), clamp_grid(cdiv(q.ny + 1, 2), 65535));
    k_apply_stencil2<<<gr, b, 0, s>>>(q, u, y, 1.0 / (3.0 * h2));
  }
  return cudaGetLastError();
}

cudaError_t launch_apply_elementwise_f64(const Geo &q, int dim, const double *u, double *y,
                                         cudaStream_t s) {
  const double h2 = q.h * q.h;
  if (dim == 3) {
    dim3 gr(cdiv(q.nx + 1, EW_TX), cdiv(q.ny + 1, EW_TY), cdiv(q.nz + 1, EW_TZ));
    if (gr.y > 65535 || gr.z > 65535) return cudaErrorInvalidConfiguration;
    k_apply_elementwise3<<<gr, 256, 0, s>>>(q, u, y, 1.0 / (12.0 * h2));
  } else {
    dim3 gr(cdiv(q.nx + 1, EW2_TX), cdiv(q.ny + 1, EW2_TY));
    if (gr.y > 65535) return cudaErrorInvalidConfiguration;
    k_apply_elementwise2<<<gr, 256, 0, s>>>(q, u, y, 1.0 / (6.0 * h2));
  }
  return cudaGetLastError();
}

cudaError_t launch_gs_sweeps_f64(const Geo &q, int dim, double *u, const double *f, int sweeps,
                                 cudaStream_t s) {
  const double g = 0.375 * q.h * q.h;
  if (q.nx < 2 || q.ny < 2 || (dim == 3 && q.nz < 2)) return cudaSuccess;  // no interior
  for (int it = 0; it < sweeps; ++it) {
    if (dim == 3) {
      // phase (py, pz): rows j = 1 + py' ... with global parity (j&1, k&1) equal to
      // the colour pair's (y, z) bits.  Global parity p of j maps to start 1 + (1-p).
      for (int ph = 0; ph < 4; ++ph) {
        const int cy = ph & 1, cz = ph >> 1;      // wanted parities of j and k
        const int sy = cy ? 0 : 1, sz = cz ? 0 : 1;  // offset from 1 with that parity
        const int64_t rows = (q.ny - 1 - sy + 1) / 2, planes = (q.nz - 1 - sz + 1) / 2;
        if (rows <= 0 || planes <= 0) continue;
        dim3 b(128, 2), gr(cdiv(q.nx - 1, 128), clamp_grid(cdiv(rows, 2), 65535),
                           clamp_grid(planes, 65535));
        k_gs_phase3<<<gr, b, 0, s>>>(q, u, f, sy, sz, g);
      }
    } else {
      for (int c = 0; c < 4; ++c) {
        const int cx = c & 1, cy = c >> 1;
        const int sx = cx ? 0 : 1, sy = cy ? 0 : 1;
        const int64_t cols = (q.nx - 1 - sx + 1) / 2, rows = (q.ny - 1 - sy + 1) / 2;
        if (cols <= 0 || rows <= 0) continue;
        dim3 b(128, 2), gr(cdiv(cols, 128), clamp_grid(cdiv(rows, 2), 65535));
        k_gs_colour2<<<gr, b, 0, s>>>(q, u, f, sx, sy, g);
      }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_jacobi_sweep_f64(const Geo &q, int dim, const double *u, const double *f,
                                    double *unew, double omega, cudaStream_t s) {
  const double h2 = q.h * q.h;
  const double w38 = omega * 0.375;
  if (dim == 3) {
    dim3 b(128, 2), gr(cdiv(q.nx + 1, 128), clamp_grid(cdiv(q.ny + 1, 2), 65535),
                       clamp_grid(q.nz + 1, 65535));
    k_jacobi3<<<gr, b, 0, s>>>(q, u, f, unew, h2, w38);
  } else {
    dim3 b(128, 2), gr(cdiv(q.nx + 1, 128), clamp_grid(cdiv(q.ny + 1, 2), 65535));
    k_jacobi2<<<gr, b, 0, s>>>(q, u, f, unew, h2, w38);
  }
  return cudaGetLastError();
}

size_t reduce_scratch_bytes() { return 16 + 2 * kReduceBlocks * sizeof(double); }

cudaError_t launch_residual_f64(const Geo &q, int dim, const double *u, const double *f,
                                double *r, double *norms2, void *scratch, cudaStream_t s) {
  // layout shared by every reduction user of this scratch: counter first, partials after
  unsigned *counter = (unsigned *)scratch;
  double *partials = (double *)((char *)scratch + 16);
  k_residual<<<kReduceBlocks, RED_THREADS, 0, s>>>(q, dim, u, f, r, norms2, partials, counter,
                                                   1.0 / (q.h * q.h));
  return cudaGetLastError();
}

}  // namespace stencil
