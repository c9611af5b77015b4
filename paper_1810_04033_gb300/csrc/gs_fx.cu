// Coloured Gauss-Seidel sweep for the 3D Q1 operator, two launches per sweep, exact
// fixed-point neighbour sums (fixed.cuh).
//
// Colour order (Section 3, "Colouring"): colour = (i&1) + 2(j&1) + 4(k&1), ascending.
// The Q1 face weight is 0, so colours 2m and 2m+1 (differing only in the x parity) are
// not coupled and can be updated together; a sweep is 4 phases over whole x-rows:
//   A = rows (j even, k even)  colours {0,1}      B = (j odd, k even)  colours {2,3}
//   C = (j even, k odd)        colours {4,5}      D = (j odd, k odd)   colours {6,7}
// A reads old B, C, D; B reads new A, old C, D; C reads new A, B, old D; D reads new
// A, B, C.  The sweep runs out of place from X into Y:
//   even launch: for every even plane z, phase A then phase B, reading X only;
//   odd launch:  for every odd plane z, phase C then phase D, reading the new even
//                planes from Y and the old D rows of plane z from X.
// Every value a phase reads is exactly the value the sequential colour order would
// read, so the result equals the in-place sweep (up to rounding of the sums).
//
// Tiling: a CTA owns an (x, y) tile of 58 x 30 vertices and a chunk of centre planes.
// For each centre plane it stages the plane's odd rows and the two neighbour planes
// (tile + 2-vertex halo) in shared memory as int64 fixed point; phase 1 (A or C) is
// computed on the tile grown by one vertex (kept in shared memory for phase 2), phase 2
// (B or D) on the tile.  Neighbour planes are shared between consecutive centre planes.
// A warp handles one row segment: lane l owns column c, forms the column sums
//   V = u(c, r-1, z) + u(c, r+1, z),  W = u(c, r, z-1) + u(c, r, z+1),
//   Q = sum of u(c, r+-1, z+-1),       P = 2(V + W) + Q,
// and the update at c is  2E + C = P(c-1) + P(c+1) + 2 Q(c)  (E: 12 edge neighbours,
// C: 8 corners), so u_new = 3/8 h^2 f + (2E + C) / 32.  Lanes 1..30 produce outputs.
//
// Fixed-point scale: a per-sweep bound on |u| tracked on the device (pre-pass for the
// first sweep, then the maximum each sweep writes), plus 4 * (3/8) h^2 max|f| for the
// growth inside a sweep.  If that bound is unusable (non-finite or extreme), the same
// kernel runs its native FP64 arithmetic instead.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fixed.cuh"
#include "internal.h"

namespace stencil {
namespace {

constexpr int GS_TX = 58, GS_TY = 30;        // output tile
constexpr int GS_SW = 64;                    // staged columns (62 used)
constexpr int GS_SH = 36;                    // staged rows (34 used, 2 zero pad rows)
constexpr int GS_THREADS = 256;
constexpr int GS_CZ = 16;                    // centre planes per CTA
constexpr int GS_NUP = GS_SH * GS_SW / GS_THREADS;             // 9 values / thread
constexpr int GS_NCE = (GS_SH / 2 * GS_SW + GS_THREADS - 1) / GS_THREADS;  // 5 (odd rows)
constexpr size_t GS_PLANE = (size_t)GS_SH * GS_SW;
constexpr size_t GS_SMEM = 3 * GS_PLANE * sizeof(long long);

struct SweepBounds {
  unsigned long long umax[3];  // max |u| of the iterate, ring indexed by sweep
  unsigned long long fmax;     // max |f| over interior vertices
};

struct Ctx {
  Geo q;
  int x0, y0;        // tile origin (vertex indices)
  int rb, e2;        // fixed-point scale
  double g;          // 3/8 h^2
  int nx, ny;        // cells (as int: planes are < 2^31 elements)
  int pitch;
};

template <bool FIX>
__device__ __forceinline__ long long enc(double v, int rb) {
  if (FIX) return fx::to_fixed(v, rb);
  return __double_as_longlong(v);
}

template <bool FIX>
__device__ __forceinline__ long long add(long long a, long long b) {
  if (FIX) return a + b;
  return __double_as_longlong(__longlong_as_double(a) + __longlong_as_double(b));
}

// In-plane offset of staged element (r, col) and whether it lies in the grid.
template <bool INNER>
__device__ __forceinline__ bool staged_at(const Ctx &c, int r, int col, int &off) {
  const int x = c.x0 - 2 + col, j = c.y0 - 2 + r;
  off = j * c.pitch + x;
  if (INNER) return col < GS_TX + 4 && r < GS_TY + 4;
  return col < GS_TX + 4 && r < GS_TY + 4 && x >= 0 && x <= c.nx && j >= 0 && j <= c.ny;
}

// Prefetch of one centre plane's odd rows (pc) and one full neighbour plane (pu).
template <bool INNER>
__device__ __forceinline__ void prefetch(const Ctx &c, const double *__restrict__ cplane,
                                         const double *__restrict__ uplane, double (&pc)[GS_NCE],
                                         double (&pu)[GS_NUP]) {
#pragma unroll
  for (int k = 0; k < GS_NCE; ++k) {
    const int idx = threadIdx.x + k * GS_THREADS;
    const int r = 2 * (idx >> 6) + 1, col = idx & 63;
    int off;
    const bool ok = idx < GS_SH / 2 * GS_SW && cplane && staged_at<INNER>(c, r, col, off);
    pc[k] = ok ? cplane[off] : 0.0;
  }
#pragma unroll
  for (int k = 0; k < GS_NUP; ++k) {
    const int idx = threadIdx.x + k * GS_THREADS;
    const int r = idx >> 6, col = idx & 63;
    int off;
    const bool ok = uplane && staged_at<INNER>(c, r, col, off);
    pu[k] = ok ? uplane[off] : 0.0;
  }
}

template <bool FIX>
__device__ __forceinline__ void commit(const Ctx &c, const double (&pc)[GS_NCE],
                                       const double (&pu)[GS_NUP], long long *ce, long long *up) {
#pragma unroll
  for (int k = 0; k < GS_NCE; ++k) {
    const int idx = threadIdx.x + k * GS_THREADS;
    if (idx < GS_SH / 2 * GS_SW) ce[(2 * (idx >> 6) + 1) * GS_SW + (idx & 63)] = enc<FIX>(pc[k], c.rb);
  }
#pragma unroll
  for (int k = 0; k < GS_NUP; ++k) up[threadIdx.x + k * GS_THREADS] = enc<FIX>(pu[k], c.rb);
}

// f values this thread needs for the two phases of one centre plane (4 rows each).
template <bool INNER>
__device__ __forceinline__ void prefetch_f(const Ctx &c, const double *__restrict__ fplane,
                                           double (&fv)[8]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg = warp & 1, grp = warp >> 1;
#pragma unroll
  for (int ph = 0; ph < 2; ++ph) {
    const int col = (ph == 0 ? 0 : 1) + 30 * seg + lane;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int r = (ph == 0 ? 2 : 3) + 8 * grp + 2 * k;
      const int x = c.x0 - 2 + col, j = c.y0 - 2 + r;
      const bool ok = fplane && lane >= 1 && lane <= 30 && x >= 1 && x < c.nx && j >= 1 && j < c.ny;
      fv[4 * ph + k] = ok ? fplane[j * c.pitch + x] : 0.0;
    }
  }
}

// One phase on the staged centre plane.  WHICH = 1: rows of parity 0 on the tile + 1
// (results also written back into the centre plane); WHICH = 2: rows of parity 1 on
// the tile.  A warp walks 4 rows of one 32-column segment, carrying the column sums of
// the shared rows from one row to the next.
template <bool FIX, bool INNER, int WHICH>
__device__ __forceinline__ void phase(const Ctx &c, long long *ce, const long long *lo,
                                      const long long *up, const double *__restrict__ xplane,
                                      double *__restrict__ yplane, const double (&fv)[8],
                                      bool zin, unsigned long long &vmax) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg = warp & 1, grp = warp >> 1;
  const int col = (WHICH == 1 ? 0 : 1) + 30 * seg + lane;
  const int r0 = (WHICH == 1 ? 2 : 3) + 8 * grp;
  const int x = c.x0 - 2 + col;
  const bool lane_out = lane >= 1 && lane <= 30 && (WHICH == 1 ? col <= 60 : col <= 59);
  const bool x_in = INNER || (x >= 0 && x <= c.nx);
  const bool x_inner = INNER || (x >= 1 && x < c.nx);
  const bool col_core = WHICH == 2 || (col >= 2 && col < 60);
  const long long *lc = lo + col, *uc = up + col;
  long long *cc = ce + col;
  long long Dm = add<FIX>(lc[(r0 - 1) * GS_SW], uc[(r0 - 1) * GS_SW]);
  long long Cm = cc[(r0 - 1) * GS_SW];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = r0 + 2 * k;
    const long long Dp = add<FIX>(lc[(r + 1) * GS_SW], uc[(r + 1) * GS_SW]);
    const long long Cp = cc[(r + 1) * GS_SW];
    const long long W = add<FIX>(lc[r * GS_SW], uc[r * GS_SW]);
    const long long V = add<FIX>(Cm, Cp);
    const long long Q = add<FIX>(Dm, Dp);
    const long long VW = add<FIX>(V, W);
    const long long P = add<FIX>(add<FIX>(VW, VW), Q);
    const long long Pm = __shfl_up_sync(0xffffffffu, P, 1);
    const long long Pp = __shfl_down_sync(0xffffffffu, P, 1);
    Dm = Dp;
    Cm = Cp;
    const int j = c.y0 - 2 + r;
    const bool row_ok = WHICH == 1 ? true : r <= GS_TY + 1;  // phase 2: last group has 3 rows
    if (!lane_out || !row_ok) continue;
    const bool in_grid = x_in && (INNER || (j >= 0 && j <= c.ny));
    if (!in_grid) continue;
    const bool inner = zin && x_inner && (INNER || (j >= 1 && j < c.ny));
    const int off = j * c.pitch + x;
    double un;
    if (inner) {
      const long long S = add<FIX>(add<FIX>(Pm, Pp), add<FIX>(Q, Q));
      if (FIX)
        un = fma(c.g, fv[(WHICH - 1) * 4 + k], fx::to_double(S, c.e2));
      else
        un = fma(__longlong_as_double(S), 0.03125, c.g * fv[(WHICH - 1) * 4 + k]);
    } else {
      un = xplane[off];  // Dirichlet value, copied
    }
    if (WHICH == 1) cc[r * GS_SW] = enc<FIX>(un, c.rb);
    if (col_core && (WHICH == 2 || r < GS_TY + 2)) {
      yplane[off] = un;
      const unsigned long long b = fx::abs_bits(un);
      vmax = b > vmax ? b : vmax;
    }
  }
}

template <bool FIX, bool INNER>
__device__ void run_half(const Ctx &c, int pz, int i0, int i1, const double *__restrict__ X,
                         const double *__restrict__ N, double *__restrict__ Y,
                         const double *__restrict__ f, long long *smem, unsigned long long &vmax) {
  const Geo &q = c.q;
  const int64_t P = q.plane;
  long long *slot[3] = {smem, smem + GS_PLANE, smem + 2 * GS_PLANE};
  int lo = 0, ce = 1, up = 2;
  double pc[GS_NCE], pu[GS_NUP], fv[8];
  // prologue: the lower neighbour of the first centre plane, then its prefetch
  {
    const int64_t z = pz + 2 * (int64_t)i0;
    double dummy[GS_NCE];
    prefetch<INNER>(c, nullptr, z >= 1 ? N + (z - 1) * P : nullptr, dummy, pu);
    commit<FIX>(c, dummy, pu, slot[ce], slot[lo]);  // ce gets zeros, overwritten below
    const bool zin = z >= 1 && z <= q.nz - 1;
    prefetch<INNER>(c, zin ? X + z * P : nullptr, z + 1 <= q.nz ? N + (z + 1) * P : nullptr, pc, pu);
    prefetch_f<INNER>(c, zin ? f + z * P : nullptr, fv);
  }
  for (int i = i0; i < i1; ++i) {
    const int64_t z = pz + 2 * (int64_t)i;
    const bool zin = z >= 1 && z <= q.nz - 1;
    commit<FIX>(c, pc, pu, slot[ce], slot[up]);
    double fcur[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) fcur[k] = fv[k];
    __syncthreads();
    if (i + 1 < i1) {  // next centre plane z + 2 and its upper neighbour z + 3
      const bool zn = z + 2 >= 1 && z + 2 <= q.nz - 1;
      prefetch<INNER>(c, zn ? X + (z + 2) * P : nullptr, z + 3 <= q.nz ? N + (z + 3) * P : nullptr,
                      pc, pu);
      prefetch_f<INNER>(c, zn ? f + (z + 2) * P : nullptr, fv);
    }
    const double *xp = X + z * P;
    double *yp = Y + z * P;
    if (zin) {
      phase<FIX, INNER, 1>(c, slot[ce], slot[lo], slot[up], xp, yp, fcur, true, vmax);
      __syncthreads();
      phase<FIX, INNER, 2>(c, slot[ce], slot[lo], slot[up], xp, yp, fcur, true, vmax);
    } else {
      // Dirichlet plane: copy the tile
      for (int idx = threadIdx.x; idx < GS_TX * GS_TY; idx += GS_THREADS) {
        const int x = c.x0 + idx % GS_TX, j = c.y0 + idx / GS_TX;
        if (x > c.nx || j > c.ny) continue;
        const double v = xp[j * c.pitch + x];
        yp[j * c.pitch + x] = v;
        const unsigned long long b = fx::abs_bits(v);
        vmax = b > vmax ? b : vmax;
      }
    }
    __syncthreads();
    // the upper neighbour becomes the next centre plane's lower neighbour
    const int t = lo;
    lo = up;
    up = t;
  }
}

__global__ void __launch_bounds__(GS_THREADS, 2)
    k_gs_half_sweep(Geo q, int pz, const double *__restrict__ X, const double *__restrict__ N,
                    double *__restrict__ Y, const double *__restrict__ f, SweepBounds *bnd,
                    int slot_read, int slot_write, int slot_clear, double g) {
  extern __shared__ long long smem[];
  __shared__ unsigned long long red[GS_THREADS / 32];
  Ctx c;
  c.q = q;
  c.x0 = (int)blockIdx.x * GS_TX;
  c.y0 = (int)blockIdx.y * GS_TY;
  c.g = g;
  c.nx = (int)q.nx;
  c.ny = (int)q.ny;
  c.pitch = (int)q.pitch;
  // bound for this sweep: max |u| of the input iterate + growth within the sweep
  const double M = __longlong_as_double((long long)bnd->umax[slot_read]);
  const double F = __longlong_as_double((long long)bnd->fmax);
  const double B = M + 4.0 * g * F;
  const bool fix = fx::bound_ok(B);
  const int R = fx::bound_exponent(B) + 1;  // one spare bit: rounding can never reach 2^R
  c.rb = 1023 + R;
  c.e2 = R - fx::FRAC - 5;  // (2E + C) / 32
  if (slot_clear >= 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0)
    bnd->umax[slot_clear] = 0ull;

  const int ncentre = q.nz >= pz ? (int)((q.nz - pz) / 2 + 1) : 0;
  const int i0 = (int)blockIdx.z * GS_CZ;
  const int i1 = i0 + GS_CZ < ncentre ? i0 + GS_CZ : ncentre;
  // interior tile: every staged vertex in the grid and every output an interior vertex
  const bool inner = c.x0 >= 2 && c.x0 + GS_TX + 1 <= c.nx && c.y0 >= 2 && c.y0 + GS_TY + 1 <= c.ny;
  unsigned long long vmax = 0ull;
  if (fix) {
    if (inner)
      run_half<true, true>(c, pz, i0, i1, X, N, Y, f, smem, vmax);
    else
      run_half<true, false>(c, pz, i0, i1, X, N, Y, f, smem, vmax);
  } else {
    run_half<false, false>(c, pz, i0, i1, X, N, Y, f, smem, vmax);
  }

  vmax = fx::warp_max_u64(vmax);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = vmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    for (int w = 0; w < GS_THREADS / 32; ++w) m = red[w] > m ? red[w] : m;
    atomicMax(&bnd->umax[slot_write], m);
  }
}

// max |u| over all vertices into umax[0], max |f| over interior vertices into fmax.
__global__ void __launch_bounds__(256) k_absmax_uf(Geo q, int dim, const double *__restrict__ u,
                                                   const double *__restrict__ f, SweepBounds *bnd) {
  __shared__ unsigned long long ru[8], rf[8];
  unsigned long long mu = 0, mf = 0;
  const int64_t nrows = (q.nz + 1) * (q.ny + 1);
  for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int64_t k = row / (q.ny + 1), j = row % (q.ny + 1);
    const bool row_inner = j > 0 && j < q.ny && (dim == 2 || (k > 0 && k < q.nz));
    const double *ur = u + k * q.plane + j * q.pitch;
    const double *fr = f + k * q.plane + j * q.pitch;
    for (int64_t i = threadIdx.x; i <= q.nx; i += blockDim.x) {
      const unsigned long long b = fx::abs_bits(ur[i]);
      mu = b > mu ? b : mu;
      if (row_inner && i > 0 && i < q.nx) {
        const unsigned long long c = fx::abs_bits(fr[i]);
        mf = c > mf ? c : mf;
      }
    }
  }
  mu = fx::warp_max_u64(mu);
  mf = fx::warp_max_u64(mf);
  if ((threadIdx.x & 31) == 0) {
    ru[threadIdx.x >> 5] = mu;
    rf[threadIdx.x >> 5] = mf;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) {
      mu = ru[w] > mu ? ru[w] : mu;
      mf = rf[w] > mf ? rf[w] : mf;
    }
    atomicMax(&bnd->umax[0], mu);
    atomicMax(&bnd->fmax, mf);
  }
}

}  // namespace

size_t gs_fx_bounds_bytes() { return sizeof(SweepBounds); }

cudaError_t launch_gs_sweeps_fx3(const Geo &q, double *u, const double *f, int sweeps,
                                 double *work, void *bounds, cudaStream_t s) {
  static bool attr_set = false;  // per process; harmless to repeat
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_gs_half_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)GS_SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (q.plane >= ((int64_t)1 << 31) - GS_SW * GS_SH) return cudaErrorInvalidValue;
  SweepBounds *bnd = (SweepBounds *)bounds;
  cudaError_t e = cudaMemsetAsync(bnd, 0, sizeof(SweepBounds), s);
  if (e != cudaSuccess) return e;
  k_absmax_uf<<<1216, 256, 0, s>>>(q, 3, u, f, bnd);
  const double g = 0.375 * q.h * q.h;
  const unsigned tx = (unsigned)((q.nx + 1 + GS_TX - 1) / GS_TX);
  const unsigned ty = (unsigned)((q.ny + 1 + GS_TY - 1) / GS_TY);
  if (ty > 65535) return cudaErrorInvalidConfiguration;
  double *cur = u, *nxt = work;
  for (int it = 0; it < sweeps; ++it) {
    const int rd = it % 3, wr = (it + 1) % 3, cl = (it + 2) % 3;
    for (int pz = 0; pz < 2; ++pz) {
      const int64_t ncentre = (q.nz - pz) / 2 + 1;
      const unsigned tz = (unsigned)((ncentre + GS_CZ - 1) / GS_CZ);
      if (tz > 65535) return cudaErrorInvalidConfiguration;
      dim3 grid(tx, ty, tz);
      k_gs_half_sweep<<<grid, GS_THREADS, GS_SMEM, s>>>(q, pz, cur, pz == 0 ? cur : nxt, nxt, f, bnd,
                                                        rd, wr, pz == 0 ? cl : -1, g);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double *t = cur;
    cur = nxt;
    nxt = t;
  }
  if (cur != u) {
    e = cudaMemcpyAsync(u, cur, (size_t)span_elems(q) * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace stencil
