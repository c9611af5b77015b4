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

constexpr int GS_TX = 58, GS_TY = 30;           // output tile
constexpr int GS_SW = 64, GS_SH = GS_TY + 4;    // staged plane: 64 columns (62 used) x 34 rows
constexpr int GS_THREADS = 256;
constexpr int GS_CZ = 16;                       // centre planes per CTA
constexpr size_t GS_SMEM = 3 * GS_SH * GS_SW * sizeof(long long);

struct Ctx {
  Geo q;
  int64_t x0, y0;
  int rb, e2;      // fixed-point scale (fix mode)
  double g;        // 3/8 h^2
};

template <bool FIX>
__device__ __forceinline__ long long enc(double v, int rb) {
  if (FIX) return fx::to_fixed(v, rb);
  return __double_as_longlong(v);
}

// Stage plane z of src into slot (rows all or odd only), zero outside the grid.
template <bool FIX>
__device__ void stage_plane(long long *slot, const double *__restrict__ src, const Ctx &c,
                            int64_t z, bool odd_rows_only) {
  const int nrows = odd_rows_only ? GS_SH / 2 : GS_SH;
  for (int idx = threadIdx.x; idx < nrows * GS_SW; idx += GS_THREADS) {
    const int r = odd_rows_only ? 2 * (idx >> 6) + 1 : (idx >> 6);
    const int col = idx & 63;
    const int64_t x = c.x0 - 2 + col, j = c.y0 - 2 + r;
    double v = 0.0;
    if (col < GS_TX + 4 && x >= 0 && x <= c.q.nx && j >= 0 && j <= c.q.ny)
      v = src[z * c.q.plane + j * c.q.pitch + x];
    slot[r * GS_SW + col] = enc<FIX>(v, c.rb);
  }
}

template <bool FIX>
__device__ __forceinline__ long long add(long long a, long long b) {
  if (FIX) return a + b;
  return __double_as_longlong(__longlong_as_double(a) + __longlong_as_double(b));
}

// One phase on centre plane z.  which = 1: rows of parity 0 on the tile + 1 (results
// also kept in shared memory); which = 2: rows of parity 1 on the tile.
template <bool FIX, int WHICH>
__device__ void phase(long long *ce, const long long *lo, const long long *up, const Ctx &c,
                      int64_t z, const double *__restrict__ X, const double *__restrict__ f,
                      double *__restrict__ Y, unsigned long long &vmax) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NROWS = WHICH == 1 ? (GS_TY / 2 + 1) : (GS_TY / 2);
  const Geo &q = c.q;
  for (int task = warp; task < NROWS * 2; task += GS_THREADS / 32) {
    const int rr = task >> 1, seg = task & 1;
    const int r = WHICH == 1 ? 2 + 2 * rr : 3 + 2 * rr;
    const int col = (WHICH == 1 ? 0 : 1) + 30 * seg + lane;
    const int64_t x = c.x0 - 2 + col, j = c.y0 - 2 + r;
    const bool out_lane = lane >= 1 && lane <= 30 && (WHICH == 1 ? col <= 60 : col <= 59);
    const bool in_grid = x >= 0 && x <= q.nx && j >= 0 && j <= q.ny;
    const bool interior = x >= 1 && x < q.nx && j >= 1 && j < q.ny;
    const bool in_core = WHICH == 2 || (col >= 2 && col < 60 && r < 32);
    const int64_t gp = z * q.plane + j * q.pitch + x;
    double fv = 0.0;
    if (out_lane && interior) fv = f[gp];
    // column sums (every lane, columns up to 63 exist in shared memory)
    const long long *cm = ce + (r - 1) * GS_SW + col, *cp = ce + (r + 1) * GS_SW + col;
    const long long *l0 = lo + r * GS_SW + col, *u0 = up + r * GS_SW + col;
    long long V = add<FIX>(cm[0], cp[0]);
    long long W = add<FIX>(l0[0], u0[0]);
    long long Q = add<FIX>(add<FIX>(l0[-GS_SW], l0[GS_SW]), add<FIX>(u0[-GS_SW], u0[GS_SW]));
    long long VW = add<FIX>(V, W);
    long long P = add<FIX>(add<FIX>(VW, VW), Q);
    const long long Pm = __shfl_up_sync(0xffffffffu, P, 1);
    const long long Pp = __shfl_down_sync(0xffffffffu, P, 1);
    if (!out_lane || !in_grid) continue;
    double un;
    if (interior) {
      const long long S = add<FIX>(add<FIX>(Pm, Pp), add<FIX>(Q, Q));
      if (FIX)
        un = fma(c.g, fv, fx::to_double(S, c.e2));
      else
        un = fma(__longlong_as_double(S), 0.03125, c.g * fv);
    } else {
      un = X[gp];  // Dirichlet value, copied
    }
    if (WHICH == 1) ce[r * GS_SW + col] = enc<FIX>(un, c.rb);
    if (in_core) {
      Y[gp] = un;
      const unsigned long long b = fx::abs_bits(un);
      vmax = b > vmax ? b : vmax;
    }
  }
}

struct SweepBounds {
  unsigned long long umax[3];  // max |u| of the iterate, ring indexed by sweep
  unsigned long long fmax;     // max |f| over interior vertices
};

template <bool FIX>
__device__ void run_half(const Ctx &c, int pz, int64_t i0, int64_t i1, const double *__restrict__ X,
                         const double *__restrict__ N, double *__restrict__ Y,
                         const double *__restrict__ f, long long *smem, unsigned long long &vmax) {
  const Geo &q = c.q;
  int lo = 0, ce = 1, up = 2;
  bool have_lower = false;
  for (int64_t i = i0; i < i1; ++i) {
    const int64_t z = pz + 2 * i;
    const bool interior_z = z >= 1 && z <= q.nz - 1;
    if (interior_z) {
      if (!have_lower) stage_plane<FIX>(smem + lo * GS_SH * GS_SW, N, c, z - 1, false);
      stage_plane<FIX>(smem + ce * GS_SH * GS_SW, X, c, z, true);
      stage_plane<FIX>(smem + up * GS_SH * GS_SW, N, c, z + 1, false);
    } else if (z + 1 <= q.nz) {
      stage_plane<FIX>(smem + up * GS_SH * GS_SW, N, c, z + 1, false);
    }
    __syncthreads();
    if (interior_z) {
      phase<FIX, 1>(smem + ce * GS_SH * GS_SW, smem + lo * GS_SH * GS_SW, smem + up * GS_SH * GS_SW,
                    c, z, X, f, Y, vmax);
      __syncthreads();
      phase<FIX, 2>(smem + ce * GS_SH * GS_SW, smem + lo * GS_SH * GS_SW, smem + up * GS_SH * GS_SW,
                    c, z, X, f, Y, vmax);
    } else {
      // Dirichlet plane: copy the tile
      for (int idx = threadIdx.x; idx < GS_TX * GS_TY; idx += GS_THREADS) {
        const int64_t x = c.x0 + idx % GS_TX, j = c.y0 + idx / GS_TX;
        if (x > q.nx || j > q.ny) continue;
        const int64_t gp = z * q.plane + j * q.pitch + x;
        const double v = X[gp];
        Y[gp] = v;
        const unsigned long long b = fx::abs_bits(v);
        vmax = b > vmax ? b : vmax;
      }
    }
    __syncthreads();
    // the upper neighbour becomes the next centre plane's lower neighbour
    const int t = lo;
    lo = up;
    up = t;
    have_lower = z + 1 <= q.nz;
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
  c.x0 = (int64_t)blockIdx.x * GS_TX;
  c.y0 = (int64_t)blockIdx.y * GS_TY;
  c.g = g;
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

  const int64_t ncentre = q.nz >= pz ? (q.nz - pz) / 2 + 1 : 0;
  const int64_t i0 = (int64_t)blockIdx.z * GS_CZ;
  const int64_t i1 = i0 + GS_CZ < ncentre ? i0 + GS_CZ : ncentre;
  unsigned long long vmax = 0ull;
  if (fix)
    run_half<true>(c, pz, i0, i1, X, N, Y, f, smem, vmax);
  else
    run_half<false>(c, pz, i0, i1, X, N, Y, f, smem, vmax);

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
