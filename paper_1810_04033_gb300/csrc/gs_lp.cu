// Coloured Gauss-Seidel for reduced-precision storage (FP32, or bf16 storage with FP32
// arithmetic), the inner solver of the iterative refinement.  Same colour phases and
// two-launch out-of-place structure as the FP64 kernel (gs_fx.cu): the even launch
// updates rows A = (j even, k even) then B = (j odd, k even) of the even planes from
// X; the odd launch updates C = (j even, k odd) then D = (j odd, k odd) of the odd
// planes, reading the new even planes from Y.  In 3D, colours 2m and 2m+1 are
// uncoupled (Q1 face weight 0), so each phase updates whole x-rows; the result equals
// the sequential colour order.  Arithmetic is FP32 (u_new = 3/8 h^2 f + (2E + C)/32);
// bf16 values are widened on load and rounded to nearest even on every store.  FP32
// arrays that TMA can stage take k_gs_lp_t (below), the rest k_gs_lp_half.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "tma.cuh"

namespace stencil {
namespace {

constexpr int LP_TX = 58, LP_TY = 30;
constexpr int LP_SW = 64, LP_SH = 36;
constexpr int LP_THREADS = 256;
constexpr int LP_CZ = 16;  // centre planes per CTA (at most)
constexpr int LP_PLANE = LP_SW * LP_SH;

template <typename S>
__device__ __forceinline__ float ld(const S *p, int64_t i);
template <>
__device__ __forceinline__ float ld<float>(const float *p, int64_t i) {
  return p[i];
}
template <>
__device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16 *p, int64_t i) {
  return __bfloat162float(p[i]);
}
template <typename S>
__device__ __forceinline__ void st(S *p, int64_t i, float v);
template <>
__device__ __forceinline__ void st<float>(float *p, int64_t i, float v) {
  p[i] = v;
}
template <>
__device__ __forceinline__ void st<__nv_bfloat16>(__nv_bfloat16 *p, int64_t i, float v) {
  p[i] = __float2bfloat16_rn(v);
}
// value as it will be stored (the next phase reads exactly what memory would hold)
template <typename S>
__device__ __forceinline__ float quant(float v);
template <>
__device__ __forceinline__ float quant<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ float quant<__nv_bfloat16>(float v) {
  return __bfloat162float(__float2bfloat16_rn(v));
}

constexpr int LP_NUP = LP_SH * LP_SW / LP_THREADS;                         // 9 values / thread
constexpr int LP_NCE = (LP_SH / 2 * LP_SW + LP_THREADS - 1) / LP_THREADS;  // 5 (odd rows)

// Raw loads of one centre plane's odd rows (pc) and one full neighbour plane (pu) of
// the tile + 2-vertex halo into registers (zeros outside the grid or for a null plane).
template <typename S>
__device__ __forceinline__ void lp_prefetch(const Geo &q, int x0, int y0, const S *cplane, const S *uplane,
                                            float (&pc)[LP_NCE], float (&pu)[LP_NUP]) {
#pragma unroll
  for (int k = 0; k < LP_NCE; ++k) {
    const int idx = threadIdx.x + k * LP_THREADS;
    const int r = 2 * (idx >> 6) + 1, col = idx & 63;
    const int64_t x = x0 - 2 + col, j = y0 - 2 + r;
    const bool ok = cplane && idx < LP_SH / 2 * LP_SW && col < LP_TX + 4 && r < LP_TY + 4 && x >= 0 &&
                    x <= q.nx && j >= 0 && j <= q.ny;
    pc[k] = ok ? ld<S>(cplane, j * q.pitch + x) : 0.0f;
  }
#pragma unroll
  for (int k = 0; k < LP_NUP; ++k) {
    const int idx = threadIdx.x + k * LP_THREADS;
    const int r = idx >> 6, col = idx & 63;
    const int64_t x = x0 - 2 + col, j = y0 - 2 + r;
    const bool ok = uplane && col < LP_TX + 4 && r < LP_TY + 4 && x >= 0 && x <= q.nx && j >= 0 && j <= q.ny;
    pu[k] = ok ? ld<S>(uplane, j * q.pitch + x) : 0.0f;
  }
}

__device__ __forceinline__ void lp_commit(const float (&pc)[LP_NCE], const float (&pu)[LP_NUP], float *ce,
                                          float *up) {
#pragma unroll
  for (int k = 0; k < LP_NCE; ++k) {
    const int idx = threadIdx.x + k * LP_THREADS;
    if (ce && idx < LP_SH / 2 * LP_SW) ce[(2 * (idx >> 6) + 1) * LP_SW + (idx & 63)] = pc[k];
  }
#pragma unroll
  for (int k = 0; k < LP_NUP; ++k) up[threadIdx.x + k * LP_THREADS] = pu[k];
}

// Right-hand sides of the two phases of one centre plane (4 rows each), 3/8 h^2 f.
template <typename S>
__device__ __forceinline__ void lp_prefetch_f(const Geo &q, int x0, int y0, const S *fplane, float g, float (&fv)[8]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg = warp & 1, grp = warp >> 1;
#pragma unroll
  for (int ph = 0; ph < 2; ++ph) {
    const int col = (ph == 0 ? 0 : 1) + 30 * seg + lane;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int r = (ph == 0 ? 2 : 3) + 8 * grp + 2 * k;
      const int64_t x = x0 - 2 + col, j = y0 - 2 + r;
      const bool ok = fplane && lane >= 1 && lane <= 30 && x >= 1 && x < q.nx && j >= 1 && j < q.ny;
      fv[4 * ph + k] = ok ? g * ld<S>(fplane, j * q.pitch + x) : 0.0f;
    }
  }
}

template <typename S, int WHICH>
__device__ void lp_phase(const Geo &q, int x0, int y0, float *ce, const float *lo, const float *up,
                         const S *xplane, S *yplane, const float (&gf)[8]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg = warp & 1, grp = warp >> 1;
  const int col = (WHICH == 1 ? 0 : 1) + 30 * seg + lane;
  const int r0 = (WHICH == 1 ? 2 : 3) + 8 * grp;
  const int64_t x = x0 - 2 + col;
  const bool lane_out = lane >= 1 && lane <= 30 && (WHICH == 1 ? col <= 60 : col <= 59);
  const bool col_core = WHICH == 2 || (col >= 2 && col < 60);
  float Dm = lo[(r0 - 1) * LP_SW + col] + up[(r0 - 1) * LP_SW + col];
  float Cm = ce[(r0 - 1) * LP_SW + col];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = r0 + 2 * k;
    const float Dp = lo[(r + 1) * LP_SW + col] + up[(r + 1) * LP_SW + col];
    const float Cp = ce[(r + 1) * LP_SW + col];
    const float W = lo[r * LP_SW + col] + up[r * LP_SW + col];
    const float V = Cm + Cp, Q = Dm + Dp;
    const float P = 2.0f * (V + W) + Q;
    const float Pm = __shfl_up_sync(0xffffffffu, P, 1);
    const float Pp = __shfl_down_sync(0xffffffffu, P, 1);
    Dm = Dp;
    Cm = Cp;
    const int64_t j = y0 - 2 + r;
    if (!lane_out || (WHICH == 2 && r > LP_TY + 1)) continue;
    if (x < 0 || x > q.nx || j < 0 || j > q.ny) continue;
    const int64_t off = j * q.pitch + x;
    float v;
    if (x >= 1 && x < q.nx && j >= 1 && j < q.ny)
      v = quant<S>(fmaf(Pm + Pp + 2.0f * Q, 0.03125f, gf[(WHICH - 1) * 4 + k]));
    else
      v = ld<S>(xplane, off);  // Dirichlet value
    if (WHICH == 1) ce[r * LP_SW + col] = v;
    if (col_core && (WHICH == 2 || r < LP_TY + 2)) st<S>(yplane, off, v);
  }
}

template <typename S>
__global__ void __launch_bounds__(LP_THREADS) k_gs_lp_half(Geo q, int pz, const S *X, const S *N, S *Y, const S *f,
                                                           float g, int cz) {
  extern __shared__ float lps[];
  auto slot = [&](int i) -> float * { return lps + i * LP_PLANE; };
  const int x0 = (int)blockIdx.x * LP_TX, y0 = (int)blockIdx.y * LP_TY;
  const int64_t ncentre = (q.nz - pz) / 2 + 1;
  const int64_t i0 = (int64_t)blockIdx.z * cz;
  const int64_t i1 = i0 + cz < ncentre ? i0 + cz : ncentre;
  int lo = 0, ce = 1, up = 2;
  float pc[LP_NCE], pu[LP_NUP], fv[8];
  {
    const int64_t z = pz + 2 * i0;
    float dummy[LP_NCE];
    lp_prefetch<S>(q, x0, y0, (const S *)nullptr, z >= 1 ? N + (z - 1) * q.plane : nullptr, dummy, pu);
    lp_commit(dummy, pu, nullptr, slot(lo));
    const bool zin = z >= 1 && z < q.nz;
    lp_prefetch<S>(q, x0, y0, zin ? X + z * q.plane : nullptr, z + 1 <= q.nz ? N + (z + 1) * q.plane : nullptr, pc,
                   pu);
    lp_prefetch_f<S>(q, x0, y0, zin ? f + z * q.plane : nullptr, g, fv);
  }
  for (int64_t i = i0; i < i1; ++i) {
    const int64_t z = pz + 2 * i;
    const bool zin = z >= 1 && z < q.nz;
    lp_commit(pc, pu, slot(ce), slot(up));
    float fcur[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) fcur[k] = fv[k];
    __syncthreads();
    if (i + 1 < i1) {  // next centre plane z + 2 and its upper neighbour z + 3
      const bool zn = z + 2 >= 1 && z + 2 < q.nz;
      lp_prefetch<S>(q, x0, y0, zn ? X + (z + 2) * q.plane : nullptr, z + 3 <= q.nz ? N + (z + 3) * q.plane : nullptr,
                     pc, pu);
      lp_prefetch_f<S>(q, x0, y0, zn ? f + (z + 2) * q.plane : nullptr, g, fv);
    }
    if (zin) {
      lp_phase<S, 1>(q, x0, y0, slot(ce), slot(lo), slot(up), X + z * q.plane, Y + z * q.plane, fcur);
      __syncthreads();
      lp_phase<S, 2>(q, x0, y0, slot(ce), slot(lo), slot(up), X + z * q.plane, Y + z * q.plane, fcur);
    } else {
      for (int idx = threadIdx.x; idx < LP_TX * LP_TY; idx += LP_THREADS) {
        const int64_t x = x0 + idx % LP_TX, j = y0 + idx / LP_TX;
        if (x > q.nx || j > q.ny) continue;
        Y[z * q.plane + j * q.pitch + x] = X[z * q.plane + j * q.pitch + x];
      }
    }
    __syncthreads();
    const int t = lo;  // the upper neighbour becomes the next centre plane's lower one
    lo = up;
    up = t;
  }
}

// ------------------------------------------------------------ TMA-staged form
// The same half sweep with the planes brought into shared memory by TMA: seven slots
// (neighbour planes z-1 and z+1 from N, centre plane z from X and its right-hand side
// from f, and the next centre plane's three new boxes in flight, issued one centre
// plane ahead), one mbarrier each, bounded waits.  Staging f with the planes keeps the
// phases free of global loads, which otherwise bound the kernel (at 257^3 the
// refinement's FP32 sweeps went from 2.34 to 1.56 s).  The staged box is 64 x 34
// values of the storage type from (x0 - HL, y0 - 2), HL chosen so that the box starts
// on a 16-byte boundary (FP32: tile 56 wide, HL = 4; bf16: tile 48 wide, HL = 8), so
// staged column c is x0 - HL + c; lane l works on the column pair 2l, 2l + 1.  Phase 1
// (even rows, the tile grown by one vertex) writes its results into the staged centre
// plane, whose other values are the old ones (Dirichlet vertices stay as they are);
// phase 2 (odd rows) reads them.
// Arithmetic as in k_gs_lp_half (FP32; bf16 widened on load, every store rounded to
// nearest even).  Used when X, N, Y and f are 16-byte aligned and the row pitch is a
// multiple of 16 bytes.  A wait that runs out sets g_lp_tma_error and the CTA leaves.
constexpr int LT_W = 64, LT_H = 34;   // staged box
constexpr int LT_TY = 30;             // output tile rows
constexpr int LT_SLOT = LT_W * LT_H;  // values per slot
constexpr int LT_NSLOT = 7;  // lo, up, centre, next up, next centre; f of the centre, f of the next
constexpr unsigned LT_WAIT = 1u << 22;
__device__ unsigned g_lp_tma_error = 0;

template <typename S>
struct LtTile;
template <>
struct LtTile<float> {
  static constexpr int TX = 56, HL = 4;
};
template <>
struct LtTile<__nv_bfloat16> {
  static constexpr int TX = 48, HL = 8;
};

template <typename S>
constexpr size_t lt_smem() {
  return (size_t)LT_NSLOT * LT_SLOT * sizeof(S) + 128;
}

struct F2 {
  float a, b;
};

__device__ __forceinline__ F2 ld2(const float *p) {
  const float2 v = *(const float2 *)p;
  return F2{v.x, v.y};
}
__device__ __forceinline__ F2 ld2(const __nv_bfloat16 *p) {
  const __nv_bfloat162 v = *(const __nv_bfloat162 *)p;
  return F2{__low2float(v), __high2float(v)};
}
__device__ __forceinline__ void st2(float *p, float a, float b) { *(float2 *)p = make_float2(a, b); }
__device__ __forceinline__ void st2(__nv_bfloat16 *p, float a, float b) {
  *(__nv_bfloat162 *)p = __floats2bfloat162_rn(a, b);
}

// One phase: WHICH 1 = even rows 2 + 4w, 4 + 4w on staged columns HL-1 .. HL+TX
// (written back into ce); WHICH 2 = odd rows 3 + 4w, 5 + 4w (up to 31) on the tile's
// columns HL .. HL+TX-1.  Y receives the tile (rows 2..31) inside the grid.
template <typename S, int WHICH, bool INNER>
__device__ __forceinline__ void lpt_phase(const Geo &q, int x0, int y0, S *ce, const S *lo, const S *up,
                                          const S *fplane, S *yplane, float g) {
  constexpr int TX = LtTile<S>::TX, HL = LtTile<S>::HL;
  constexpr int c0 = WHICH == 1 ? HL - 1 : HL, c1 = WHICH == 1 ? HL + TX : HL + TX - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col = 2 * lane;
  const int r0 = (WHICH == 1 ? 2 : 3) + 4 * warp;
  const int64_t xa = x0 - HL + col;
  const bool va = col >= c0 && col <= c1, vb = col + 1 >= c0 && col + 1 <= c1;
  const bool core = col >= HL && col + 1 <= HL + TX - 1;
  const bool xa_in = INNER || (xa >= 1 && xa < q.nx), xb_in = INNER || (xa + 1 >= 1 && xa + 1 < q.nx);
  const bool xa_ok = INNER || (xa >= 0 && xa <= q.nx), xb_ok = INNER || (xa + 1 >= 0 && xa + 1 <= q.nx);
  const S *lc = lo + col, *uc = up + col;
  S *cc = ce + col;
  F2 Dm = ld2(lc + (r0 - 1) * LT_W), Dum = ld2(uc + (r0 - 1) * LT_W);
  Dm = F2{Dm.a + Dum.a, Dm.b + Dum.b};
  F2 Cm = ld2(cc + (r0 - 1) * LT_W);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int r = r0 + 2 * k;
    if (WHICH == 2 && r > 31) break;  // warp-uniform
    const int64_t j = y0 - 2 + r;
    const bool jin = INNER || (j >= 1 && j < q.ny);
    const bool ja = va && xa_in && jin, jb = vb && xb_in && jin;
    // right-hand side 3/8 h^2 f (FP32) from the staged f plane (used where updated)
    const F2 fv = ld2(fplane + r * LT_W + col);
    const F2 gf{g * fv.a, g * fv.b};
    const F2 l1 = ld2(lc + (r + 1) * LT_W), u1 = ld2(uc + (r + 1) * LT_W);
    const F2 Dp{l1.a + u1.a, l1.b + u1.b};
    const F2 Cp = ld2(cc + (r + 1) * LT_W);
    const F2 l0 = ld2(lc + r * LT_W), u0 = ld2(uc + r * LT_W);
    const F2 W{l0.a + u0.a, l0.b + u0.b};
    const F2 V{Cm.a + Cp.a, Cm.b + Cp.b}, Q{Dm.a + Dp.a, Dm.b + Dp.b};
    const F2 P{2.0f * (V.a + W.a) + Q.a, 2.0f * (V.b + W.b) + Q.b};
    const float Pl = __shfl_up_sync(0xffffffffu, P.b, 1);
    const float Pr = __shfl_down_sync(0xffffffffu, P.a, 1);
    Dm = Dp;
    Cm = Cp;
    const F2 old = ld2(cc + r * LT_W);
    F2 nw = old;
    if (ja) nw.a = quant<S>(fmaf(Pl + P.b + 2.0f * Q.a, 0.03125f, gf.a));
    if (jb) nw.b = quant<S>(fmaf(P.a + Pr + 2.0f * Q.b, 0.03125f, gf.b));
    if (WHICH == 1) st2(cc + r * LT_W, nw.a, nw.b);
    const bool jok = INNER || (j >= 0 && j <= q.ny);
    const bool rcore = r >= 2 && r <= 31;
    const bool wa = core && rcore && jok && xa_ok, wb = core && rcore && jok && xb_ok;
    S *yrow = yplane + j * q.pitch;
    if (wa && wb) {
      st2(yrow + xa, nw.a, nw.b);
    } else {
      if (wa) st<S>(yrow, xa, nw.a);
      if (wb) st<S>(yrow, xa + 1, nw.b);
    }
  }
}

template <typename S>
__global__ void __launch_bounds__(LP_THREADS) k_gs_lp_t(Geo q, int pz, S *Y, const S *f, float g, int cz,
                                                        const __grid_constant__ CUtensorMap mapX,
                                                        const __grid_constant__ CUtensorMap mapN,
                                                        const __grid_constant__ CUtensorMap mapF) {
  constexpr int TX = LtTile<S>::TX, HL = LtTile<S>::HL;
  extern __shared__ unsigned char lt_raw[];
  __shared__ __align__(8) uint64_t bars[LT_NSLOT];
  __shared__ int fail;
  S *sm = (S *)(((uintptr_t)lt_raw + 127) & ~(uintptr_t)127);
  auto slot = [&](int i) -> S * { return sm + i * LT_SLOT; };
  const int x0 = (int)blockIdx.x * TX, y0 = (int)blockIdx.y * LT_TY;
  // every computed vertex (staged columns HL-1 .. HL+TX, rows 2..32) interior
  const bool inner = x0 - 1 >= 1 && x0 + TX <= q.nx - 1 && y0 >= 1 && y0 + 30 <= q.ny - 1;
  const int64_t ncentre = (q.nz - pz) / 2 + 1;
  const int64_t i0 = (int64_t)blockIdx.z * cz;
  const int64_t i1 = i0 + cz < ncentre ? i0 + cz : ncentre;
  if (threadIdx.x == 0) {
    for (int i = 0; i < LT_NSLOT; ++i) mbar_init(&bars[i], 1);
    fail = 0;
    fence_mbar_init();
    fence_proxy_async();
  }
  __syncthreads();
  unsigned ph = 0, pend = 0;
  int sl_lo = 0, sl_up = 1, sl_ce = 2, sl_nup = 3, sl_nce = 4, sl_fc = 5, sl_fn = 6;
  auto issue = [&](int s, const CUtensorMap *m, int64_t z) {
    pend |= 1u << s;
    if (threadIdx.x == 0) {
      fence_proxy_async();  // earlier generic accesses to the slot before the TMA writes it
      tma_load_plane(slot(s), m, x0 - HL, y0 - 2, (int)z, &bars[s], LT_SLOT * sizeof(S));
    }
  };
  auto wait = [&](int s) {
    if (!mbar_wait(&bars[s], (ph >> s) & 1u, LT_WAIT)) {
      atomicExch(&fail, 1);  // the load stays pending
      return;
    }
    ph ^= 1u << s;
    pend &= ~(1u << s);
  };
  bool ok = i0 < i1;
  if (ok) {
    const int64_t z = pz + 2 * i0;
    issue(sl_lo, &mapN, z - 1);
    issue(sl_up, &mapN, z + 1);
    issue(sl_ce, &mapX, z);
    issue(sl_fc, &mapF, z);
    if (i0 + 1 < i1) {
      issue(sl_nce, &mapX, z + 2);
      issue(sl_nup, &mapN, z + 3);
      issue(sl_fn, &mapF, z + 2);
    }
    wait(sl_lo);
  }
  for (int64_t i = i0; i < i1 && ok; ++i) {
    const int64_t z = pz + 2 * i;
    wait(sl_ce);
    wait(sl_up);
    wait(sl_fc);
    __syncthreads();
    if (fail) {
      ok = false;
      break;
    }
    S *yp = Y + z * q.plane;
    if (z >= 1 && z < q.nz) {
      const S *fp = slot(sl_fc);
      if (inner) {
        lpt_phase<S, 1, true>(q, x0, y0, slot(sl_ce), slot(sl_lo), slot(sl_up), fp, yp, g);
        __syncthreads();
        lpt_phase<S, 2, true>(q, x0, y0, slot(sl_ce), slot(sl_lo), slot(sl_up), fp, yp, g);
      } else {
        lpt_phase<S, 1, false>(q, x0, y0, slot(sl_ce), slot(sl_lo), slot(sl_up), fp, yp, g);
        __syncthreads();
        lpt_phase<S, 2, false>(q, x0, y0, slot(sl_ce), slot(sl_lo), slot(sl_up), fp, yp, g);
      }
    } else {
      // Dirichlet plane: carry the tile through
      const S *cs = slot(sl_ce);
      for (int idx = threadIdx.x; idx < TX * LT_TY; idx += LP_THREADS) {
        const int64_t x = x0 + idx % TX, j = y0 + idx / TX;
        if (x > q.nx || j > q.ny) continue;
        yp[j * q.pitch + x] = cs[(j - y0 + 2) * LT_W + (x - x0 + HL)];
      }
    }
    __syncthreads();  // every access to the freed slots is done
    const int t_lo = sl_lo, t_ce = sl_ce, t_fc = sl_fc;
    sl_lo = sl_up;
    sl_up = sl_nup;
    sl_ce = sl_nce;
    sl_fc = sl_fn;
    sl_nup = t_lo;
    sl_nce = t_ce;
    sl_fn = t_fc;
    if (i + 2 < i1) {
      issue(sl_nce, &mapX, z + 4);
      issue(sl_nup, &mapN, z + 5);
      issue(sl_fn, &mapF, z + 4);
    }
  }
  if (!ok && i0 < i1) {  // wait once more (bounded) for every load still in flight
    for (int s = 0; s < LT_NSLOT; ++s)
      if (pend & (1u << s)) mbar_wait(&bars[s], (ph >> s) & 1u, LT_WAIT);
    if (threadIdx.x == 0) atomicExch(&g_lp_tma_error, 1u);
  }
}

}  // namespace

template <typename S>
static cudaError_t gs_lp_sweeps(const Geo &q, S *u, const S *f, int sweeps, S *work, cudaStream_t s) {
  static PerDeviceOnce attr;
  const size_t smem = 3 * (size_t)LP_PLANE * sizeof(float);
  {
    cudaError_t e = set_smem_limit_once(attr, k_gs_lp_half<S>, smem);
    if (e != cudaSuccess) return e;
  }
  const float g = (float)(0.375 * q.h * q.h);
  const unsigned tx = (unsigned)((q.nx + LP_TX) / LP_TX), ty = (unsigned)((q.ny + LP_TY) / LP_TY);
  if (ty > 65535) return cudaErrorInvalidConfiguration;
  S *X = u, *Y = work;
  // the TMA-staged kernel where the arrays allow it
  CUtensorMap mu, mw, mf;
  const bool tma = ((uintptr_t)f % 16) == 0 && tma_plane_map_elem(q, u, (int)sizeof(S), LT_W, LT_H, &mu) &&
                   tma_plane_map_elem(q, work, (int)sizeof(S), LT_W, LT_H, &mw) &&
                   tma_plane_map_elem(q, f, (int)sizeof(S), LT_W, LT_H, &mf);
  if (tma) {
    static PerDeviceOnce attr_t;
    cudaError_t e = set_smem_limit_once(attr_t, k_gs_lp_t<S>, lt_smem<S>());
    if (e != cudaSuccess) return e;
  }
  constexpr int TTX = LtTile<S>::TX;
  const unsigned ttx = (unsigned)((q.nx + TTX) / TTX), tty = (unsigned)((q.ny + LT_TY) / LT_TY);
  if (tty > 65535) return cudaErrorInvalidConfiguration;
  for (int it = 0; it < sweeps; ++it) {
    for (int pz = 0; pz < 2; ++pz) {
      const int64_t ncentre = (q.nz - pz) / 2 + 1;
      if (tma) {
        const int cz = z_chunk((int64_t)ttx * tty, ncentre, LP_CZ, 2, 4);
        const unsigned tz = (unsigned)((ncentre + cz - 1) / cz);
        const CUtensorMap &mx = X == u ? mu : mw, &my = Y == u ? mu : mw;
        k_gs_lp_t<S><<<dim3(ttx, tty, tz), LP_THREADS, lt_smem<S>(), s>>>(q, pz, Y, f, g, cz, mx,
                                                                          pz == 0 ? mx : my, mf);
      } else {
        const int cz = z_chunk((int64_t)tx * ty, ncentre, LP_CZ, 2, 8);
        const unsigned tz = (unsigned)((ncentre + cz - 1) / cz);
        k_gs_lp_half<S><<<dim3(tx, ty, tz), LP_THREADS, smem, s>>>(q, pz, X, pz == 0 ? X : Y, Y, f, g, cz);
      }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    S *t = X;
    X = Y;
    Y = t;
  }
  if (X != u) return cudaMemcpyAsync(u, X, (size_t)span_elems(q) * sizeof(S), cudaMemcpyDeviceToDevice, s);
  return cudaSuccess;
}

cudaError_t launch_gs_sweeps_f32_3d(const Geo &q, float *u, const float *f, int sweeps, float *work,
                                    cudaStream_t s) {
  return gs_lp_sweeps<float>(q, u, f, sweeps, work, s);
}

cudaError_t launch_gs_sweeps_bf16_3d(const Geo &q, void *u, const void *f, int sweeps, void *work,
                                     cudaStream_t s) {
  return gs_lp_sweeps<__nv_bfloat16>(q, (__nv_bfloat16 *)u, (const __nv_bfloat16 *)f, sweeps,
                                     (__nv_bfloat16 *)work, s);
}

}  // namespace stencil

namespace stencil {

// The TMA wait flag of this file's kernels (1 once a bounded wait ran out); cleared on
// request.  Synchronous.
cudaError_t tma_wait_flag_gs_lp(unsigned *value, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(value, g_lp_tma_error, sizeof(unsigned));
  if (e == cudaSuccess && clear && *value) {
    const unsigned zero = 0u;
    e = cudaMemcpyToSymbol(g_lp_tma_error, &zero, sizeof(unsigned));
  }
  return e;
}

}  // namespace stencil
