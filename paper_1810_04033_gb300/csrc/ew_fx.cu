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
// A CTA owns 60 x 32 (x, y) output vertices and a chunk of 32 vertex planes.  It streams
// cell layers k = z0-1, z0, ...: layer k lies between vertex planes k and k+1, whose
// values sit in shared memory (with a 1-vertex halo), together with two int64
// accumulator planes.  The race of the scatter is resolved by colours: the z parity by
// processing layers in order, the y parity by two passes per layer separated by
// barriers, the x parity inside each warp (neighbouring cells' shared vertices are
// combined through a shuffle, see scatter_layer).  After layer k, vertex plane k has
// received all 8 contributions and is written out.  The fixed-point reference is the
// per-CTA monotone scheme of ops_fx.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fixed.cuh"
#include "internal.h"

namespace stencil {
namespace {

constexpr int ET_X = 60, ET_Y = 32;        // output vertices per tile
constexpr int ES_W = 64, ES_H = ET_Y + 2;  // staged vertex plane: 64 columns (62 used) x 34 rows
constexpr int E_THREADS = 256;
constexpr int E_CZ = 32;
constexpr int E_PER = (ES_W * ES_H + E_THREADS - 1) / E_THREADS;
constexpr int E_PLANE = ES_W * ES_H;
constexpr size_t E_SMEM = 4 * (size_t)E_PLANE * sizeof(long long);
constexpr int R_MIN = -900, R_MAX = 1000;

struct EwArgs {
  Geo q;
  const double *u;
  double *y;
  double scale;  // 1 / (12 h^2)
  int cz;        // planes per CTA
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

__device__ __forceinline__ void prefetch_vplane(double (&v)[E_PER], const Geo &q, const double *src,
                                                int64_t z, int x0, int y0) {
  const bool zok = z >= 0 && z <= q.nz;
  const double *p = src + (zok ? z : 0) * q.plane;
#pragma unroll
  for (int k = 0; k < E_PER; ++k) {
    const int idx = threadIdx.x + k * E_THREADS;
    const int r = idx >> 6, col = idx & 63;
    const int x = x0 - 1 + col, j = y0 - 1 + r;
    const bool ok = zok && idx < E_PLANE && col < ET_X + 2 && x >= 0 && x <= q.nx && j >= 0 && j <= q.ny;
    v[k] = ok ? p[(int64_t)j * q.pitch + x] : 0.0;
  }
}

__device__ __forceinline__ int cta_max_exponent(const double (&v)[E_PER], int *red) {
  unsigned m = 0;
#pragma unroll
  for (int k = 0; k < E_PER; ++k) {
    const unsigned e = (unsigned)(fx::dbits(v[k]) >> 52) & 0x7ffu;
    m = e > m ? e : m;
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (int)m;
  __syncthreads();
  int r = 0;
#pragma unroll
  for (int w = 0; w < E_THREADS / 32; ++w) r = red[w] > r ? red[w] : r;
  return r;
}

// Cell layer k (between vertex planes k and k+1).  A warp takes one row of 32
// consecutive cells (local cells lcx = 30 seg + lane); each lane computes its cell's 8
// contributions: with bottom-face values b_i (plane k) and top-face values t_i (plane
// k+1), i = 0 (x,y), 1 (x+1,y), 2 (x,y+1), 3 (x+1,y+1), and face sums Sb, St,
//   12 (K u)_{b_i} = 4 b_i - b_{i^3} + t_i - St,   12 (K u)_{t_i} = 4 t_i - t_{i^3} + b_i - Sb.
// The right-hand vertices' contributions move to the next lane by a shuffle (the two x
// colours of the row meet in registers), so each output lane adds the sums for its own
// vertex column into the shared accumulators of vertex rows y and y+1 of both planes.
// Cell rows of one y parity share no vertex row: the two y colours are separate
// passes with a barrier between them; layers run in z order.
template <bool FIX>
__device__ void scatter_layer(const Geo &q, int64_t k, int x0, int y0, const long long *ulo,
                              const long long *uhi, long long *alo, long long *ahi) {
  if (k < 0 || k >= q.nz) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int py = 0; py < 2; ++py) {
    const int lcy0 = ((y0 - 1) & 1) == py ? 0 : 1;
    // tasks: (cell row, segment); rows lcy = lcy0, lcy0 + 2, ... < ET_Y + 1
    const int nrows = (ET_Y + 1 - lcy0 + 1) / 2;
    for (int task = warp; task < 2 * nrows; task += E_THREADS / 32) {
      const int lcy = lcy0 + 2 * (task >> 1), seg = task & 1;
      const int lcx = 30 * seg + lane;  // local cell; covers vertex columns lcx, lcx+1
      const int cx = x0 - 1 + lcx, cy = y0 - 1 + lcy;
      const int i0 = lcy * ES_W + lcx, i1 = i0 + ES_W;
      const long long b0 = ulo[i0], b2 = ulo[i1], t0 = uhi[i0], t2 = uhi[i1];
      const long long b1 = __shfl_down_sync(0xffffffffu, b0, 1);
      const long long b3 = __shfl_down_sync(0xffffffffu, b2, 1);
      const long long t1 = __shfl_down_sync(0xffffffffu, t0, 1);
      const long long t3 = __shfl_down_sync(0xffffffffu, t2, 1);
      const bool cell = lane <= 30 && cx >= 0 && cx < q.nx && cy >= 0 && cy < q.ny;
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
      }
      // the left neighbour's right-hand contributions land on this lane's column
      const long long lb1 = __shfl_up_sync(0xffffffffu, cb1, 1);
      const long long lb3 = __shfl_up_sync(0xffffffffu, cb3, 1);
      const long long lt1 = __shfl_up_sync(0xffffffffu, ct1, 1);
      const long long lt3 = __shfl_up_sync(0xffffffffu, ct3, 1);
      if (lane < 1 || lane > 30) continue;
      alo[i0] = add<FIX>(alo[i0], add<FIX>(cb0, lb1));
      alo[i1] = add<FIX>(alo[i1], add<FIX>(cb2, lb3));
      ahi[i0] = add<FIX>(ahi[i0], add<FIX>(ct0, lt1));
      ahi[i1] = add<FIX>(ahi[i1], add<FIX>(ct2, lt3));
    }
    __syncthreads();
  }
}

template <bool FIX>
__device__ void write_plane(const EwArgs &a, int64_t z, int x0, int y0, int R, const long long *acc) {
  const Geo &q = a.q;
  if (z < 0 || z > q.nz) return;
  double *out = a.y + z * q.plane;
  const bool zin = z >= 1 && z < q.nz;
  for (int idx = threadIdx.x; idx < ET_X * ET_Y; idx += E_THREADS) {
    const int lx = idx % ET_X, ly = idx / ET_X;
    const int x = x0 + lx, j = y0 + ly;
    if (x > q.nx || j > q.ny) continue;
    const bool inner = zin && x >= 1 && x < q.nx && j >= 1 && j < q.ny;
    const long long s = acc[(ly + 1) * ES_W + lx + 1];
    double yv = 0.0;
    if (inner) yv = FIX ? fx::to_double(s, R - fx::FRAC) * a.scale : __longlong_as_double(s) * a.scale;
    out[(int64_t)j * q.pitch + x] = yv;
  }
}

__global__ void __launch_bounds__(E_THREADS, 3) k_apply_elementwise_fx3(EwArgs a) {
  extern __shared__ long long smem[];
  __shared__ int red[E_THREADS / 32];
  const Geo &q = a.q;
  const int x0 = (int)blockIdx.x * ET_X, y0 = (int)blockIdx.y * ET_Y;
  const int64_t zs = (int64_t)blockIdx.z * a.cz;
  const int64_t ze = zs + a.cz < q.nz + 1 ? zs + a.cz : q.nz + 1;
  auto slot = [&](int i) -> long long * { return smem + i * E_PLANE; };
  int ulo = 0, uhi = 1, alo = 2, ahi = 3;
  bool fix = true;
  int R = R_MIN;
  double v[E_PER];

  for (int idx = threadIdx.x; idx < 4 * E_PLANE; idx += E_THREADS) smem[idx] = 0;
  __syncthreads();

  // Admit a prefetched vertex plane into slot dst; rescale or switch to FP64 as needed
  // (live slots: the other staged plane and both accumulators).
  auto admit = [&](int dst) {
    const int em = cta_max_exponent(v, red);
    if (fix && em != 0) {
      const int Rp = em - 1022 + 1;
      const int Rn = Rp > R ? Rp : R;
      if (em == 2047 || Rp > R_MAX || (Rp < R_MIN && R == R_MIN)) {
        for (int idx = threadIdx.x; idx < 4 * E_PLANE; idx += E_THREADS)
          if (idx / E_PLANE != dst)
            smem[idx] = __double_as_longlong(fx::to_double(smem[idx], R - fx::FRAC));
        fix = false;
      } else if (Rn > R && Rp >= R_MIN) {
        const int d = Rn - R;
        for (int idx = threadIdx.x; idx < 4 * E_PLANE; idx += E_THREADS)
          if (idx / E_PLANE != dst) smem[idx] = d < 63 ? (smem[idx] >> d) : (smem[idx] >> 63);
        R = Rn;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < E_PER; ++k) {
      const int idx = threadIdx.x + k * E_THREADS;
      if (idx < E_PLANE) slot(dst)[idx] = fix ? fx::to_fixed(v[k], 1023 + R) : __double_as_longlong(v[k]);
    }
  };

  // cell layers zs-1 .. ze-1; layer k needs vertex planes k and k+1
  prefetch_vplane(v, q, a.u, zs - 1, x0, y0);
  admit(ulo);
  prefetch_vplane(v, q, a.u, zs, x0, y0);
  for (int64_t k = zs - 1; k < ze; ++k) {
    admit(uhi);  // vertex plane k + 1
    __syncthreads();
    if (k + 2 <= ze) prefetch_vplane(v, q, a.u, k + 2, x0, y0);
    if (fix)
      scatter_layer<true>(q, k, x0, y0, slot(ulo), slot(uhi), slot(alo), slot(ahi));
    else
      scatter_layer<false>(q, k, x0, y0, slot(ulo), slot(uhi), slot(alo), slot(ahi));
    // vertex plane k now holds all contributions
    if (k >= zs) {
      if (fix)
        write_plane<true>(a, k, x0, y0, R, slot(alo));
      else
        write_plane<false>(a, k, x0, y0, R, slot(alo));
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < E_PLANE; idx += E_THREADS) slot(alo)[idx] = 0;
    int t = ulo;
    ulo = uhi;
    uhi = t;
    t = alo;
    alo = ahi;
    ahi = t;
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_apply_elementwise_fx3(const Geo &q, const double *u, double *y, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_apply_elementwise_fx3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)E_SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int64_t txy = ((q.nx + ET_X) / ET_X) * ((q.ny + ET_Y) / ET_Y);
  const int cz = z_chunk(txy, q.nz + 1, E_CZ, 4, 3);
  const dim3 g((unsigned)((q.nx + ET_X) / ET_X), (unsigned)((q.ny + ET_Y) / ET_Y), (unsigned)((q.nz + cz) / cz));
  if (g.y > 65535 || g.z > 65535) return cudaErrorInvalidConfiguration;
  EwArgs a;
  a.q = q;
  a.u = u;
  a.y = y;
  a.scale = 1.0 / (12.0 * q.h * q.h);
  a.cz = cz;
  k_apply_elementwise_fx3<<<g, E_THREADS, E_SMEM, s>>>(a);
  return cudaGetLastError();
}

}  // namespace stencil
