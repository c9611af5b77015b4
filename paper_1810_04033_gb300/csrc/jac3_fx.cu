// Multi-sweep damped Jacobi for the 3D Q1 operator (0 < omega <= 1), the iterate kept in
// HBM as int64 fixed point between the sweeps of one call at the scale shared by the
// whole grid and tracked on the device (sweep_bounds.cuh), 3/8 h^2 f precomputed once
// per call as fixed point (GF):
//   u' = u + omega (3/8 h^2 f + (2E + C) / 32 - u),
// E and C the sums of the 12 edge and 8 corner neighbours (face weights 0), omega
// applied as the integer product of Omega.  |u'| <= max |u| + omega 3/8 h^2 max |f|,
// within the bound of sweep_bounds.cuh.  If the plan rules out fixed point, every
// sweep of the call computes in FP64 on FP64 buffers instead (the formula of the
// single-step kernel, ops_fx.cu).
//
// Planes come into four shared-memory slots by TMA (cp.async.bulk.tensor, one
// mbarrier each, bounded waits), two planes ahead of the one being computed; a plane
// already at this sweep's scale is used as it arrives, an FP64 plane (first sweep) or
// a scale change is converted in place.  A CTA owns a 60 x 32 (x, y) tile and a chunk
// of planes; lane l works on the staged column pair 2l, 2l + 1 (the box starts at
// x0 - 2) with the column sums of ops_fx.cu.  A wait that runs out sets
// g_jac3_tma_error and the CTA leaves.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fixed.cuh"
#include "internal.h"
#include "sweep_bounds.cuh"
#include "tma.cuh"

namespace stencil {
namespace {

constexpr int J3_TX = 60, J3_TY = 32;  // output tile
constexpr int J3_W = 64, J3_H = 34;    // staged box
constexpr int J3_THREADS = 256;
constexpr int J3_SLOT = J3_W * J3_H;
constexpr int J3_CZ = 32;
constexpr size_t J3_SMEM = 4 * (size_t)J3_SLOT * sizeof(long long) + 128;
constexpr unsigned J3_WAIT = 1u << 22;
__device__ unsigned g_jac3_tma_error = 0;

enum { JF64 = 0, JFXP = 1 };  // storage format: FP64, or int64 fixed point

struct L2 {
  long long a, b;
};

template <bool FIXA>
__device__ __forceinline__ long long add(long long a, long long b) {
  if (FIXA) return a + b;
  return __double_as_longlong(__longlong_as_double(a) + __longlong_as_double(b));
}

template <bool FIXA>
__device__ __forceinline__ L2 add2(const L2 &x, const L2 &y) {
  return L2{add<FIXA>(x.a, y.a), add<FIXA>(x.b, y.b)};
}

__device__ __forceinline__ L2 lds2(const long long *p) {
  const longlong2 v = *(const longlong2 *)p;
  return L2{v.x, v.y};
}

struct J3Args {
  Geo q;
  void *Y;
  const double *f;       // FP64 path
  const long long *GF;   // fixed path
  SweepBounds *bnd;
  int sweep, sweeps, cz;
  double g;              // 3/8 h^2
  double c1, c2;         // FP64 path: omega 3/8 h^2, -omega 3/8 / 12
  long long Wq;
  bool write_bnd;
};

// One plane of outputs from the staged planes lo, ce, up (staged column c = x0 - 2 + c,
// row r = y0 - 1 + r): warp w walks rows 1 + 4w .. 4 + 4w.
template <bool FIXA, int YF, bool INNER>
__device__ __forceinline__ void jac3_plane(const J3Args &a, int64_t z, int x0, int y0, int R, int dfr,
                                           const Omega &om, const long long *lo, const long long *ce,
                                           const long long *up, long long &vmax) {
  const Geo &q = a.q;
  const int nx = (int)q.nx, ny = (int)q.ny, pitch = (int)q.pitch;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col = 2 * lane, r0 = 1 + 4 * warp;
  const int xa = x0 - 2 + col;
  const bool zin = z >= 1 && z < q.nz;
  const bool lane_out = lane >= 1 && lane <= 30;
  const bool oka = INNER || xa <= nx, okb = INNER || xa + 1 <= nx;
  const bool ina = INNER || (xa >= 1 && xa < nx), inb = INNER || (xa + 1 >= 1 && xa + 1 < nx);
  // right-hand sides of the warp's 4 rows (GF: fixed point; f: FP64 bits)
  L2 rhs[4];
  {
    const long long *src = FIXA ? a.GF + z * q.plane : (const long long *)a.f + z * q.plane;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int j = y0 - 1 + r0 + k;
      const bool jin = lane_out && zin && (INNER || (j >= 1 && j < ny));
      rhs[k] = L2{0ll, 0ll};
      if (jin && ina && inb) {
        rhs[k] = lds2(src + (int64_t)j * pitch + xa);  // global, 16-byte aligned
      } else if (jin) {
        if (ina) rhs[k].a = src[(int64_t)j * pitch + xa];
        if (inb) rhs[k].b = src[(int64_t)j * pitch + xa + 1];
      }
    }
  }
  const long long *lc = lo + col, *uc = up + col, *cc = ce + col;
  L2 Cm = lds2(cc + (r0 - 1) * J3_W), Cc = lds2(cc + r0 * J3_W);
  L2 Wm = add2<FIXA>(lds2(lc + (r0 - 1) * J3_W), lds2(uc + (r0 - 1) * J3_W));
  L2 Wc = add2<FIXA>(lds2(lc + r0 * J3_W), lds2(uc + r0 * J3_W));
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = r0 + k;
    const L2 Cp = lds2(cc + (r + 1) * J3_W);
    const L2 Wp = add2<FIXA>(lds2(lc + (r + 1) * J3_W), lds2(uc + (r + 1) * J3_W));
    const L2 V = add2<FIXA>(Cm, Cp);
    const L2 Q = add2<FIXA>(Wm, Wp);
    const L2 VW = add2<FIXA>(V, Wc);
    const L2 P = add2<FIXA>(add2<FIXA>(VW, VW), Q);
    const long long Pl = __shfl_up_sync(0xffffffffu, P.b, 1);
    const long long Pr = __shfl_down_sync(0xffffffffu, P.a, 1);
    const L2 Cu = Cc;
    Cm = Cc;
    Cc = Cp;
    Wm = Wc;
    Wc = Wp;
    const int j = y0 - 1 + r;
    if (!lane_out || (!INNER && j > ny)) continue;
    const bool jin = zin && (INNER || (j >= 1 && j < ny));
    const bool ia = jin && ina, ib = jin && inb;
    L2 nw = Cu;  // Dirichlet values carried
    if (ia || ib) {
      const long long Sa = add<FIXA>(add<FIXA>(Pl, P.b), add<FIXA>(Q.a, Q.a));  // 2E + C
      const long long Sb = add<FIXA>(add<FIXA>(P.a, Pr), add<FIXA>(Q.b, Q.b));
      if (FIXA) {
        if (ia) nw.a = Cu.a + om((rhs[k].a >> dfr) + (Sa >> 5) - Cu.a);
        if (ib) nw.b = Cu.b + om((rhs[k].b >> dfr) + (Sb >> 5) - Cu.b);
      } else {
        auto upd = [&](long long c, long long S, long long fbits) {
          const double Td = fma(32.0, __longlong_as_double(c), -__longlong_as_double(S));
          return __double_as_longlong(
              fma(a.c2, Td, fma(a.c1, __longlong_as_double(fbits), __longlong_as_double(c))));
        };
        if (ia) nw.a = upd(Cu.a, Sa, rhs[k].a);
        if (ib) nw.b = upd(Cu.b, Sb, rhs[k].b);
      }
    }
    const bool wa = oka && (ia || a.write_bnd), wb = okb && (ib || a.write_bnd);
    if (!(wa || wb)) continue;
    long long ya = nw.a, yb = nw.b;
    if (FIXA && YF == JF64) {  // last sweep: only updated vertices are written
      ya = __double_as_longlong(fx::to_double_cvt(nw.a, R - fx::FRAC));
      yb = __double_as_longlong(fx::to_double_cvt(nw.b, R - fx::FRAC));
    }
    long long *yrow = (long long *)a.Y + z * q.plane + (int64_t)j * pitch;
    if (wa && wb) {
      *(longlong2 *)(yrow + xa) = make_longlong2(ya, yb);
    } else if (wa) {
      yrow[xa] = ya;
    } else {
      yrow[xa + 1] = yb;
    }
    auto mag = [&](long long v) -> long long {
      return FIXA ? (v < 0 ? -v : v) : (long long)fx::abs_bits(__longlong_as_double(v));
    };
    if (wa) vmax = max(vmax, mag(nw.a));
    if (wb) vmax = max(vmax, mag(nw.b));
  }
}

template <bool FIXA, int XF, int YF, bool INNER>
__device__ void jac3_run(const J3Args &a, const CUtensorMap *map, int64_t zs, int64_t ze, int x0, int y0, int R,
                         int dx, int dfr, long long *sm, uint64_t *bars, int *fail, long long &vmax) {
  auto slot = [&](int i) -> long long * { return sm + i * J3_SLOT; };
  const Omega om(a.Wq);
  unsigned ph = 0, pend = 0;
  int lo = 0, ce = 1, up = 2, nx = 3;
  auto issue = [&](int s, int64_t z) {
    pend |= 1u << s;
    if (threadIdx.x == 0) {
      fence_proxy_async();  // earlier generic accesses to the slot before the TMA writes it
      tma_load_plane(slot(s), map, x0 - 2, y0 - 1, (int)z, &bars[s], J3_SLOT * 8);
    }
  };
  // wait for slot s and bring it to this sweep's representation; false if a wait ran out
  auto admit = [&](int s) -> bool {
    if (mbar_wait(&bars[s], (ph >> s) & 1u, J3_WAIT)) {
      ph ^= 1u << s;
      pend &= ~(1u << s);
    } else {
      atomicExch(fail, 1);
    }
    __syncthreads();
    if (*fail) return false;
    if (FIXA && (XF == JF64 || dx != 0)) {
      long long *p = slot(s);
      for (int idx = threadIdx.x; idx < J3_SLOT; idx += J3_THREADS)
        p[idx] = XF == JF64 ? fx::to_fixed(__longlong_as_double(p[idx]), 1023 + R) : shr_any(p[idx], dx);
    }
    return true;
  };
  issue(lo, zs - 1);
  issue(ce, zs);
  issue(up, zs + 1);
  bool ok = admit(lo) && admit(ce);
  for (int64_t z = zs; z < ze && ok; ++z) {
    ok = admit(up);
    __syncthreads();
    if (!ok) break;
    if (z + 2 <= ze) issue(nx, z + 2);
    jac3_plane<FIXA, YF, INNER>(a, z, x0, y0, R, dfr, om, slot(lo), slot(ce), slot(up), vmax);
    __syncthreads();
    const int t = lo;
    lo = ce;
    ce = up;
    up = nx;
    nx = t;
  }
  if (!ok) {  // wait once more (bounded) for every load still in flight
    for (int s = 0; s < 4; ++s)
      if (pend & (1u << s)) mbar_wait(&bars[s], (ph >> s) & 1u, J3_WAIT);
  }
}

template <int XF, int YF>
__global__ void __launch_bounds__(J3_THREADS, 3) k_jac3_sweep(J3Args a, const __grid_constant__ CUtensorMap map) {
  extern __shared__ unsigned char j3_raw[];
  __shared__ __align__(8) uint64_t bars[4];
  __shared__ long long red[J3_THREADS / 32];
  __shared__ int fail;
  long long *sm = (long long *)(((uintptr_t)j3_raw + 127) & ~(uintptr_t)127);
  const Geo &q = a.q;
  const int x0 = (int)blockIdx.x * J3_TX, y0 = (int)blockIdx.y * J3_TY;
  const int64_t zs = (int64_t)blockIdx.z * a.cz;
  const int64_t ze = zs + a.cz < q.nz + 1 ? zs + a.cz : q.nz + 1;
  const Plan plan = make_plan(a.bnd, a.g, a.sweeps);
  const int R = sweep_R(a.bnd, a.sweep % 4, a.g);
  const int Rx = a.sweep > 0 ? sweep_R(a.bnd, (a.sweep + 3) % 4, a.g) : R;
  const int dx = XF == JFXP ? R - Rx : 0, df = R - plan.Rf;
  const int dfr = df < 63 ? df : 63;
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0)
    a.bnd->umax[(a.sweep + 2) % 4] = 0ull;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(&bars[i], 1);
    fail = 0;
    fence_mbar_init();
    fence_proxy_async();
  }
  __syncthreads();
  // every output (x0 .. x0+59, y0 .. y0+31) an interior vertex and every staged vertex
  // inside the grid
  const bool inner = x0 - 2 >= 0 && x0 + 61 <= q.nx - 1 && y0 - 1 >= 0 && y0 + 32 <= q.ny - 1;
  long long vmax = 0;
  if (plan.fix) {
    if (inner)
      jac3_run<true, XF, YF, true>(a, &map, zs, ze, x0, y0, R, dx, dfr, sm, bars, &fail, vmax);
    else
      jac3_run<true, XF, YF, false>(a, &map, zs, ze, x0, y0, R, dx, dfr, sm, bars, &fail, vmax);
  } else {
    jac3_run<false, JF64, JF64, false>(a, &map, zs, ze, x0, y0, R, 0, dfr, sm, bars, &fail, vmax);
  }
  __syncthreads();
  if (fail && threadIdx.x == 0) atomicExch(&g_jac3_tma_error, 1u);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long w = __shfl_xor_sync(0xffffffffu, vmax, o);
    vmax = w > vmax ? w : vmax;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = vmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long m = 0;
    for (int w = 0; w < J3_THREADS / 32; ++w) m = red[w] > m ? red[w] : m;
    const unsigned long long mb =
        plan.fix ? fx::abs_bits(fx::to_double(m, R - fx::FRAC) * (1.0 + 0x1p-50)) : (unsigned long long)m;
    atomicMax(&a.bnd->umax[(a.sweep + 1) % 4], mb);
  }
}

template <int XF, int YF>
cudaError_t launch_j3(const J3Args &a, const CUtensorMap &map, dim3 grid, cudaStream_t s) {
  static PerDeviceOnce attr;
  {
    cudaError_t e = set_smem_limit_once(attr, k_jac3_sweep<XF, YF>, J3_SMEM);
    if (e) return e;
  }
  k_jac3_sweep<XF, YF><<<grid, J3_THREADS, J3_SMEM, s>>>(a, map);
  return cudaGetLastError();
}

}  // namespace

// Multi-sweep damped Jacobi, 3D, 0 < omega <= 1.  A: u-sized buffer (the caller's
// work array); scratch: 2 u-sized buffers (second ping-pong buffer and GF); bounds:
// gs_fx_bounds_bytes().  The result ends in u; u's boundary is never written.  Arrays
// that TMA cannot stage (base not 16-byte aligned, odd pitch) take the single-step
// kernel sweep by sweep instead.
cudaError_t launch_jacobi_sweeps_fx3(const Geo &q, double *u, const double *f, int sweeps, double omega, double *A,
                                     double *scratch, void *bounds, cudaStream_t s) {
  const int64_t span = span_elems(q);
  void *B = scratch;
  long long *GF = (long long *)(scratch + span);
  CUtensorMap mu, ma, mb;
  const bool tma = sweeps >= 2 && ((uintptr_t)f % 16) == 0 && ((uintptr_t)scratch % 16) == 0 &&
                   tma_plane_map(q, u, J3_W, J3_H, &mu) && tma_plane_map(q, A, J3_W, J3_H, &ma) &&
                   tma_plane_map(q, B, J3_W, J3_H, &mb);
  if (!tma) {
    double *a = u, *b = A;
    for (int it = 0; it < sweeps; ++it) {
      cudaError_t e = launch_jacobi_fx3(q, a, f, b, omega, s);
      if (e) return e;
      double *t = a;
      a = b;
      b = t;
    }
    return a == u ? cudaSuccess : cudaMemcpyAsync(u, a, (size_t)span * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  cudaError_t e = launch_gs_prepass(q, 3, u, f, GF, bounds, sweeps, s);
  if (e) return e;
  J3Args a{};
  a.q = q;
  a.f = f;
  a.GF = GF;
  a.bnd = (SweepBounds *)bounds;
  a.sweeps = sweeps;
  a.g = 0.375 * q.h * q.h;
  a.c1 = omega * a.g;
  a.c2 = -omega * 0.375 / 12.0;
  a.Wq = (long long)llrint(omega * 0x1p62);
  const int64_t tx = (q.nx + J3_TX) / J3_TX, ty = (q.ny + J3_TY) / J3_TY;
  a.cz = tuned_chunk(tuning_lookup(STENCIL_CALL_SMOOTH_JACOBI, q), z_chunk(tx * ty, q.nz + 1, J3_CZ, 4, 3), 4, J3_CZ);
  const dim3 grid((unsigned)tx, (unsigned)ty, (unsigned)((q.nz + a.cz) / a.cz));
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
  const CUtensorMap *X = &mu;
  for (int it = 0; it < sweeps && !e; ++it) {
    const bool first = it == 0, last = it == sweeps - 1;
    a.sweep = it;
    a.Y = last ? (void *)u : (it % 2 == 0 ? (void *)A : B);
    a.write_bnd = !last;  // the caller's u: its Dirichlet values were never overwritten
    if (first)
      e = launch_j3<JF64, JFXP>(a, *X, grid, s);
    else if (!last)
      e = launch_j3<JFXP, JFXP>(a, *X, grid, s);
    else
      e = launch_j3<JFXP, JF64>(a, *X, grid, s);
    X = it % 2 == 0 ? &ma : &mb;
  }
  return e;
}

}  // namespace stencil

namespace stencil {

// The TMA wait flag of this file's kernels (1 once a bounded wait ran out); cleared on
// request.  Synchronous.
cudaError_t tma_wait_flag_jac3(unsigned *value, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(value, g_jac3_tma_error, sizeof(unsigned));
  if (e == cudaSuccess && clear && *value) {
    const unsigned zero = 0u;
    e = cudaMemcpyToSymbol(g_jac3_tma_error, &zero, sizeof(unsigned));
  }
  return e;
}

}  // namespace stencil
