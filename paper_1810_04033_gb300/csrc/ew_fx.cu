// Element-wise (cell-wise) 3D Q1 apply on the integer pipes: every cell computes
// K_e u_e and adds it into its 8 vertices, with the 2^3 cell colours resolving the
// races of the scatter (Section 2: cell-wise weighted sums; Section 3: colouring).
//
// Per cell, 12 K_e/h (the Q1 element matrix scaled to integers: 4 on the diagonal, 0
// for vertices differing in one coordinate, -1 otherwise) gives, for local vertex w,
//   12 (K u_e)_w = 5 u_w + F_w - T,   F_w = sum of the 3 face-adjacent vertices of w,
//   T = sum of all 8 vertex values of the cell,
// evaluated exactly in int64 fixed point (fixed.cuh), so the accumulated vertex sums
// do not depend on the order of the additions.  y = sum / (12 h^2) on interior
// vertices, 0 on the boundary.
//
// The scatter runs in registers, one warp per column of cells (layout below): the z
// colours are the cell layers processed in order, the y colours the cell rows processed
// one after the other, and the x colours meet through shuffles, each vertex column
// being owned by one lane.  After layer k, vertex plane k has received all 8
// contributions and is written out.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fixed.cuh"
#include "internal.h"

namespace stencil {
namespace {

struct EwArgs {
  Geo q;
  const double *u;
  double *y;
  double scale;  // 1 / (12 h^2)
  int cz;        // output planes per warp
};

template <bool FIX>
__device__ __forceinline__ long long add(long long a, long long b) {
  if (FIX) return a + b;
  return __double_as_longlong(__longlong_as_double(a) + __longlong_as_double(b));
}

template <bool FIX>
__device__ __forceinline__ long long sub(long long a, long long b) {
  if (FIX) return a - b;
  return __double_as_longlong(__longlong_as_double(a) - __longlong_as_double(b));
}

template <bool FIX>
__device__ __forceinline__ long long times4(long long a) {
  if (FIX) return a << 2;
  return __double_as_longlong(4.0 * __longlong_as_double(a));
}

// ------------------------------------------------------------ register-streaming form
// A warp owns 32 consecutive cell columns (lanes 1..30 own the output vertex columns),
// R vertex rows y and a chunk of planes, and streams the cell layers k in z order with
// everything in registers: the vertex values of planes k and k+1 for rows j0-1..j0+R,
// the sums of plane k (contributions of layers k-1 and k) and the partial sums of plane
// k+1 (layer k).  Per layer it forms the R+1 cell rows' 8 contributions per cell; the
// right-hand vertices' shares reach the next lane by a shuffle (the x colours meet in
// registers), the y colours are the cell rows processed one after the other, the z
// colours the layers in order; after layer k, plane k has all 8 shares and is written.
// The fixed-point reference is per warp and only grows (as in the 2D kernels); a warp
// that meets a value outside the fixed-point range switches to FP64 at a layer start.
constexpr int S3_R = 4;          // output vertex rows per warp
constexpr int S3_CZ = 32;        // output planes per warp (at most)
constexpr int S3_THREADS = 128;
constexpr int S3_RMIN = -900, S3_RMAX = 1000;

struct Ew3Lane {
  int64_t x;
  bool xok, xin, cell_lane, out_lane;
  int lane;
  long long bk[S3_R + 2];  // plane k, rows j0-1 .. j0+R
  long long acc[S3_R];     // plane k rows j0 .. j0+R-1
  int R;
  bool fix;
};

__device__ __forceinline__ unsigned bexp(double v) { return (unsigned)(fx::dbits(v) >> 52) & 0x7ffu; }

__device__ __forceinline__ long long shr_pos(long long v, int d) { return d >= 63 ? (v >> 63) : (v >> d); }

// Layers k0 .. z1-1 of the warp's column; returns the first layer not done (the warp
// switched to FP64) or z1.
template <bool FIX>
__device__ __forceinline__ int64_t ew3_layers(const EwArgs &a, Ew3Lane &L, int64_t j0, int64_t z0, int64_t z1,
                                              int64_t k0) {
  const Geo &q = a.q;
  const double *ucol = a.u + (L.xok ? L.x : 0);
  auto load_plane = [&](double (&v)[S3_R + 2], int64_t z) {
#pragma unroll
    for (int c = 0; c < S3_R + 2; ++c) {
      const int64_t j = j0 - 1 + c;
      v[c] = (L.xok && z >= 0 && z <= q.nz && j >= 0 && j <= q.ny) ? ucol[z * q.plane + j * q.pitch] : 0.0;
    }
  };
  double qn[S3_R + 2];
  load_plane(qn, k0 + 1);
  for (int64_t k = k0; k < z1; ++k) {
    double tr[S3_R + 2];
#pragma unroll
    for (int c = 0; c < S3_R + 2; ++c) tr[c] = qn[c];
    if (FIX) {
      unsigned em = 0;
#pragma unroll
      for (int c = 0; c < S3_R + 2; ++c) em = max(em, bexp(tr[c]));
      em = __reduce_max_sync(0xffffffffu, em);
      if (em != 0) {
        const int Rp = (int)em - 1022 + 1;
        if (em == 2047 || Rp > S3_RMAX || (Rp < S3_RMIN && L.R == S3_RMIN)) {
#pragma unroll
          for (int c = 0; c < S3_R + 2; ++c) L.bk[c] = __double_as_longlong(fx::to_double(L.bk[c], L.R - fx::FRAC));
#pragma unroll
          for (int r = 0; r < S3_R; ++r) L.acc[r] = __double_as_longlong(fx::to_double(L.acc[r], L.R - fx::FRAC));
          L.fix = false;
          return k;  // redo this layer in FP64 (it reloads plane k+1)
        }
        if (Rp > L.R) {
          const int d = Rp - L.R;
#pragma unroll
          for (int c = 0; c < S3_R + 2; ++c) L.bk[c] = shr_pos(L.bk[c], d);
#pragma unroll
          for (int r = 0; r < S3_R; ++r) L.acc[r] = shr_pos(L.acc[r], d);
          L.R = Rp;
        }
      }
    }
    if (k + 1 < z1) load_plane(qn, k + 2);
    long long tk[S3_R + 2];
#pragma unroll
    for (int c = 0; c < S3_R + 2; ++c) tk[c] = FIX ? fx::to_fixed(tr[c], 1023 + L.R) : __double_as_longlong(tr[c]);
    long long part[S3_R];
#pragma unroll
    for (int r = 0; r < S3_R; ++r) part[r] = FIX ? 0ll : __double_as_longlong(0.0);
    if (k >= 0 && k < q.nz) {
#pragma unroll
      for (int c = 0; c <= S3_R; ++c) {
        const int64_t cj = j0 - 1 + c;
        const long long b0 = L.bk[c], b2 = L.bk[c + 1], t0 = tk[c], t2 = tk[c + 1];
        const long long b1 = __shfl_down_sync(0xffffffffu, b0, 1);
        const long long b3 = __shfl_down_sync(0xffffffffu, b2, 1);
        const long long t1 = __shfl_down_sync(0xffffffffu, t0, 1);
        const long long t3 = __shfl_down_sync(0xffffffffu, t2, 1);
        const bool cell = L.cell_lane && cj >= 0 && cj < q.ny;
        long long cb0 = 0, cb1 = 0, cb2 = 0, cb3 = 0, ct0 = 0, ct1 = 0, ct2 = 0, ct3 = 0;
        if (cell) {
          const long long Sb = add<FIX>(add<FIX>(b0, b1), add<FIX>(b2, b3));
          const long long St = add<FIX>(add<FIX>(t0, t1), add<FIX>(t2, t3));
          cb0 = add<FIX>(sub<FIX>(times4<FIX>(b0), b3), sub<FIX>(t0, St));
          cb1 = add<FIX>(sub<FIX>(times4<FIX>(b1), b2), sub<FIX>(t1, St));
          cb2 = add<FIX>(sub<FIX>(times4<FIX>(b2), b1), sub<FIX>(t2, St));
          cb3 = add<FIX>(sub<FIX>(times4<FIX>(b3), b0), sub<FIX>(t3, St));
          ct0 = add<FIX>(sub<FIX>(times4<FIX>(t0), t3), sub<FIX>(b0, Sb));
          ct1 = add<FIX>(sub<FIX>(times4<FIX>(t1), t2), sub<FIX>(b1, Sb));
          ct2 = add<FIX>(sub<FIX>(times4<FIX>(t2), t1), sub<FIX>(b2, Sb));
          ct3 = add<FIX>(sub<FIX>(times4<FIX>(t3), t0), sub<FIX>(b3, Sb));
        } else if (!FIX) {
          cb0 = cb1 = cb2 = cb3 = ct0 = ct1 = ct2 = ct3 = __double_as_longlong(0.0);
        }
        // the left neighbour's right-hand shares land on this lane's column
        long long lb1 = __shfl_up_sync(0xffffffffu, cb1, 1), lb3 = __shfl_up_sync(0xffffffffu, cb3, 1);
        long long lt1 = __shfl_up_sync(0xffffffffu, ct1, 1), lt3 = __shfl_up_sync(0xffffffffu, ct3, 1);
        if (L.lane == 0) lb1 = lb3 = lt1 = lt3 = FIX ? 0ll : __double_as_longlong(0.0);
        if (c >= 1) {  // vertex row cj (index c-1)
          L.acc[c - 1] = add<FIX>(L.acc[c - 1], add<FIX>(cb0, lb1));
          part[c - 1] = add<FIX>(part[c - 1], add<FIX>(ct0, lt1));
        }
        if (c < S3_R) {  // vertex row cj + 1 (index c)
          L.acc[c] = add<FIX>(L.acc[c], add<FIX>(cb2, lb3));
          part[c] = add<FIX>(part[c], add<FIX>(ct2, lt3));
        }
      }
    }
    if (k >= z0 && k <= q.nz && L.out_lane) {
      const bool zin = k >= 1 && k < q.nz;
      double *out = a.y + k * q.plane + L.x;
      // scale 2^(R-52) / (12 h^2), exact power-of-two scaling of a.scale
      const double sc = FIX ? a.scale * fx::pow2d(L.R - fx::FRAC) : a.scale;
#pragma unroll
      for (int r = 0; r < S3_R; ++r) {
        const int64_t j = j0 + r;
        if (j > q.ny) break;
        const bool inner = zin && L.xin && j >= 1 && j < q.ny;
        double yv = 0.0;
        if (inner) yv = (FIX ? __ll2double_rn(L.acc[r]) : __longlong_as_double(L.acc[r])) * sc;
        out[j * q.pitch] = yv;
      }
    }
#pragma unroll
    for (int r = 0; r < S3_R; ++r) L.acc[r] = part[r];
#pragma unroll
    for (int c = 0; c < S3_R + 2; ++c) L.bk[c] = tk[c];
  }
  return z1;
}

__global__ void __launch_bounds__(S3_THREADS) k_apply_elementwise_s3(EwArgs a) {
  const Geo &q = a.q;
  const int lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * (S3_THREADS / 32) + (threadIdx.x >> 5);
  const int64_t nseg = (q.nx + 30) / 30, njc = (q.ny + S3_R) / S3_R;
  const int64_t seg = gw % nseg, rest = gw / nseg;
  const int64_t jc = rest % njc, zc = rest / njc;
  const int64_t z0 = zc * a.cz;
  if (z0 > q.nz) return;
  const int64_t z1 = z0 + a.cz < q.nz + 1 ? z0 + a.cz : q.nz + 1;
  const int64_t j0 = jc * S3_R;
  Ew3Lane L;
  L.lane = lane;
  L.x = seg * 30 + lane - 1;
  L.xok = L.x >= 0 && L.x <= q.nx;
  L.xin = L.x >= 1 && L.x < q.nx;
  L.cell_lane = lane <= 30 && L.x >= 0 && L.x < q.nx;
  L.out_lane = lane >= 1 && lane <= 30 && L.xok;
  L.R = S3_RMIN;
  L.fix = true;
  // plane z0-1 (the first layer's bottom face) and no contributions yet
  {
    const double *ucol = a.u + (L.xok ? L.x : 0);
    double v[S3_R + 2];
    unsigned em = 0;
#pragma unroll
    for (int c = 0; c < S3_R + 2; ++c) {
      const int64_t j = j0 - 1 + c, z = z0 - 1;
      v[c] = (L.xok && z >= 0 && j >= 0 && j <= q.ny) ? ucol[z * q.plane + j * q.pitch] : 0.0;
      em = max(em, bexp(v[c]));
    }
    em = __reduce_max_sync(0xffffffffu, em);
    if (em != 0) {
      const int Rp = (int)em - 1022 + 1;
      if (em == 2047 || Rp > S3_RMAX || Rp < S3_RMIN)
        L.fix = false;
      else
        L.R = Rp;
    }
#pragma unroll
    for (int c = 0; c < S3_R + 2; ++c) L.bk[c] = L.fix ? fx::to_fixed(v[c], 1023 + L.R) : __double_as_longlong(v[c]);
#pragma unroll
    for (int r = 0; r < S3_R; ++r) L.acc[r] = L.fix ? 0ll : __double_as_longlong(0.0);
  }
  int64_t k = z0 - 1;
  if (L.fix) k = ew3_layers<true>(a, L, j0, z0, z1, k);
  if (k < z1) ew3_layers<false>(a, L, j0, z0, z1, k);
}

}  // namespace

cudaError_t launch_apply_elementwise_fx3(const Geo &q, const double *u, double *y, cudaStream_t s) {
  const int64_t nseg = (q.nx + 30) / 30, njc = (q.ny + S3_R) / S3_R;
  const int cz = z_chunk(nseg * njc, q.nz + 1, S3_CZ, 4, 64);
  const int64_t nzc = (q.nz + cz) / cz;
  const int64_t warps = nseg * njc * nzc;
  const int64_t blocks = (warps + S3_THREADS / 32 - 1) / (S3_THREADS / 32);
  if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
  EwArgs a;
  a.q = q;
  a.u = u;
  a.y = y;
  a.scale = 1.0 / (12.0 * q.h * q.h);
  a.cz = cz;
  k_apply_elementwise_s3<<<(unsigned)blocks, S3_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace stencil
