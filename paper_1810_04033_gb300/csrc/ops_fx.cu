// Out-of-place 3D Q1 operations on the integer pipes: assembled apply y = A u, one
// damped Jacobi sweep, and the residual r = f - A u with its norms.
//
// All three need 12 S u = 32 u - (2E + C) (E: sum of the 12 edge neighbours, C: sum of
// the 8 corner neighbours; face weights are 0), computed exactly in int64 fixed point
// (fixed.cuh) with the same column-sum scheme as the Gauss-Seidel kernel:
//   V = u(r-1) + u(r+1) in plane z, W = u(z-1) + u(z+1) in row r, Q = the four
//   diagonal (r+-1, z+-1) values, P = 2(V + W) + Q, and 2E + C = P(c-1) + P(c+1) + 2Q(c).
// A CTA owns a 60 x 32 (x, y) tile and a chunk of 32 planes; it streams z with three
// staged planes (tile + 1-vertex halo) in shared memory and prefetches the next plane
// into registers while it computes the current one (k_ops3), or has TMA bring the
// planes two ahead into four slots (k_ops3t, used when the array allows it).
//
// Fixed-point scale without a pre-pass: the CTA keeps a reference exponent R that only
// grows.  Each newly staged plane's largest exponent is reduced over the CTA first; if
// it exceeds R, the two planes already staged are shifted right to the new R.  If a
// plane holds a non-finite value or the magnitudes leave [2^-900, 2^1000], the CTA
// converts its staged planes to FP64 and finishes in native FP64 arithmetic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fixed.cuh"
#include "internal.h"
#include "tma.cuh"

namespace stencil {
namespace {

constexpr int OT_X = 60, OT_Y = 32;          // outputs per tile
constexpr int OS_W = 64, OS_H = OT_Y + 2;    // staged plane: 64 columns (62 used) x 34 rows
constexpr int O_THREADS = 256;
constexpr int O_CZ = 32;                     // output planes per CTA (at most)
constexpr int O_PER = (OS_W * OS_H + O_THREADS - 1) / O_THREADS;  // prefetched values / thread
constexpr size_t O_SMEM = 3 * OS_H * OS_W * sizeof(long long);
constexpr int R_MIN = -900, R_MAX = 1000;

enum { OP_APPLY = 0, OP_JACOBI = 1, OP_RESIDUAL = 2 };

// Per operation: convert the fixed-point result with the FP64 pipe (true) or with
// integer instructions (false), whichever measured faster.
constexpr bool OPS3_CVT[3] = {true, false, false};

// Per operation: the TMA-staged kernel computes on column pairs (compute_plane2, true)
// or one column per lane (compute_plane), whichever measured faster.
constexpr bool OPS3_PAIRS[3] = {true, false, false};

// On column pairs with OPS3_CVT: the odd-x column converts with integer instructions
// (true), a quarter of the conversions' FP64-pipe work moved to the integer pipes.
constexpr bool OPS3_SPLIT[3] = {true, false, false};

struct OpArgs {
  Geo q;
  const double *u;
  const double *f;
  double *out;       // y, u_new or r (may be null for the residual)
  double c1, c2;     // apply: c1 = 1/(12 h^2); jacobi: c1 = omega 3/8 h^2, c2 = -omega 3/8 / 12;
                     // residual: c1 = -1/(12 h^2)
  double *partials;  // residual: 2 per CTA
  unsigned *counter; // residual: CTAs finished
  double *norms2;    // residual: [sum r^2, sum f^2]
  int out_kind;      // residual: 0 = r in FP64, 1 = FP32, 2 = bf16 (FP64 -> FP32 -> bf16)
  int cz;            // output planes per CTA
  bool v16;          // f and out (FP64) 16-byte aligned with an even pitch: pair accesses
};

__device__ __forceinline__ void prefetch_plane(double (&v)[O_PER], const Geo &q, const double *src,
                                               int64_t z, int64_t x0, int64_t y0) {
#pragma unroll
  for (int k = 0; k < O_PER; ++k) {
    const int idx = threadIdx.x + k * O_THREADS;
    const int r = idx >> 6, col = idx & 63;
    const int64_t x = x0 - 1 + col, j = y0 - 1 + r;
    double val = 0.0;
    if (idx < OS_W * OS_H && col < OT_X + 2 && z >= 0 && z <= q.nz && x >= 0 && x <= q.nx &&
        j >= 0 && j <= q.ny)
      val = src[z * q.plane + j * q.pitch + x];
    v[k] = val;
  }
}

// Largest biased exponent among the prefetched values of the whole CTA (0: all zero or
// subnormal; 2047: a non-finite value).
__device__ __forceinline__ int cta_max_exponent(const double (&v)[O_PER], int *red) {
  unsigned m = 0;
#pragma unroll
  for (int k = 0; k < O_PER; ++k) {
    const unsigned e = (unsigned)(fx::dbits(v[k]) >> 52) & 0x7ffu;
    m = e > m ? e : m;
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (int)m;
  __syncthreads();
  int r = 0;
#pragma unroll
  for (int w = 0; w < O_THREADS / 32; ++w) r = red[w] > r ? red[w] : r;
  return r;
}

template <bool FIX>
__device__ __forceinline__ long long add(long long a, long long b) {
  if (FIX) return a + b;
  return __double_as_longlong(__longlong_as_double(a) + __longlong_as_double(b));
}

// Outputs of plane z from the staged planes lo (z-1), ce (z), up (z+1).  Warp w owns
// column segment w & 1 and the 8 consecutive rows 1 + 8 (w >> 1) ... ; walking down the
// rows it carries W = lo + up and the centre-plane values, so each output needs three
// new shared-memory loads: with W(r) = lo(r) + up(r),
//   V = ce(r-1) + ce(r+1),  Q = W(r-1) + W(r+1),  P = 2 (V + W(r)) + Q.
template <bool FIX, int OP, bool INNER>
__device__ __forceinline__ void compute_plane(const OpArgs &a, int64_t z, int x0, int y0, int R,
                                              const long long *lo, const long long *ce,
                                              const long long *up, double &rr, double &ff) {
  const Geo &q = a.q;
  const int nx = (int)q.nx, ny = (int)q.ny, pitch = (int)q.pitch;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col = 30 * (warp & 1) + lane, r0 = 1 + 8 * (warp >> 1);
  const int x = x0 - 1 + col;
  const bool zin = z >= 1 && z < q.nz;
  const bool lane_out = lane >= 1 && lane <= 30 && (INNER || x <= nx);
  const bool x_inner = INNER || (x >= 1 && x < nx);
  const double *fp = a.f ? a.f + z * q.plane : nullptr;
  const double *up_src = a.u + z * q.plane;
  double *outp = a.out ? a.out + z * q.plane : nullptr;
  double fv[8], uv[8];
  if (OP != OP_APPLY) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int j = y0 - 1 + r0 + k;
      const bool ok = lane_out && (INNER || j <= ny);
      const bool inner = ok && zin && x_inner && (INNER || (j >= 1 && j < ny));
      const int off = j * pitch + x;
      fv[k] = inner ? fp[off] : 0.0;
      uv[k] = (OP == OP_JACOBI && ok) ? up_src[off] : 0.0;
    }
  }
  const int e2 = R - fx::FRAC;
  // CVT: 12 S u is converted by the FP64 pipe and scaled by its term's factor times
  // 2^e2; otherwise by fx::to_double on the integer pipe (the same bits either way)
  constexpr bool CVT = OPS3_CVT[OP];
  const double cf = OP == OP_JACOBI ? a.c2 : a.c1;
  const double sc = FIX && CVT ? cf * fx::pow2d(e2) : cf;
  const long long *lc = lo + col, *uc = up + col, *cc = ce + col;
  long long Cm = cc[(r0 - 1) * OS_W], Cc = cc[r0 * OS_W];
  long long Wm = add<FIX>(lc[(r0 - 1) * OS_W], uc[(r0 - 1) * OS_W]);
  long long Wc = add<FIX>(lc[r0 * OS_W], uc[r0 * OS_W]);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int r = r0 + k;
    const long long Cp = cc[(r + 1) * OS_W];
    const long long Wp = add<FIX>(lc[(r + 1) * OS_W], uc[(r + 1) * OS_W]);
    const long long V = add<FIX>(Cm, Cp);
    const long long Q = add<FIX>(Wm, Wp);
    const long long VW = add<FIX>(V, Wc);
    const long long P = add<FIX>(add<FIX>(VW, VW), Q);
    const long long Pm = __shfl_up_sync(0xffffffffu, P, 1);
    const long long Pp = __shfl_down_sync(0xffffffffu, P, 1);
    const long long Cu = Cc;
    Cm = Cc;
    Cc = Cp;
    Wm = Wc;
    Wc = Wp;
    const int j = y0 - 1 + r;
    if (!lane_out || (!INNER && j > ny)) continue;
    const int off = j * pitch + x;
    const bool inner = zin && x_inner && (INNER || (j >= 1 && j < ny));
    double Td = 0.0;  // 32 u - (2E + C) = 12 (S u); Td * sc is its term
    if (inner) {
      const long long S = add<FIX>(add<FIX>(Pm, Pp), add<FIX>(Q, Q));
      if (FIX) {
        const long long T = 32 * Cu - S;
        Td = CVT ? __ll2double_rn(T) : fx::to_double(T, e2);
      } else {
        Td = fma(32.0, __longlong_as_double(Cu), -__longlong_as_double(S));
      }
    }
    if (OP == OP_APPLY) {
      outp[off] = inner ? Td * sc : 0.0;
    } else if (OP == OP_JACOBI) {
      outp[off] = inner ? fma(sc, Td, fma(a.c1, fv[k], uv[k])) : uv[k];
    } else {
      const double rv = inner ? fma(sc, Td, fv[k]) : 0.0;
      if (a.out) {
        const int64_t e = z * q.plane + off;  // element index
        if (a.out_kind == 0)
          a.out[e] = rv;
        else if (a.out_kind == 1)
          ((float *)a.out)[e] = (float)rv;
        else
          ((__nv_bfloat16 *)a.out)[e] = __float2bfloat16_rn((float)rv);
      }
      if (inner) {
        rr = fma(rv, rv, rr);
        ff = fma(fv[k], fv[k], ff);
      }
    }
  }
}

// Lane-pair form of compute_plane for the TMA-staged kernel, whose staged column c is
// x0 - 2 + c: lane l owns the columns 2l and 2l + 1 (xa even, xb = xa + 1) and lanes
// 1..30 produce outputs, so every shared-memory access moves a 16-byte pair and one
// shuffle per direction serves two outputs.  Warp w walks the 4 rows 1 + 4w ..
// 4 + 4w.  With P as in compute_plane,
//   2E + C at xa = (P(xa - 1) + P(xb)) + 2 Q(xa),  at xb = (P(xa) + P(xb + 1)) + 2 Q(xb),
// P(xa - 1) being the left lane's P(xb) and P(xb + 1) the right lane's P(xa).
struct LL2 {
  long long a, b;
};

template <bool FIX>
__device__ __forceinline__ LL2 add2(const LL2 &x, const LL2 &y) {
  return LL2{add<FIX>(x.a, y.a), add<FIX>(x.b, y.b)};
}

__device__ __forceinline__ LL2 lds2(const long long *p) {
  const longlong2 v = *(const longlong2 *)p;
  return LL2{v.x, v.y};
}

// A pair of FP64 values of row pointer p at columns xa, xb (zeros where not wanted).
__device__ __forceinline__ void ldg2(const double *p, int xa, bool wa, bool wb, bool v16, double &va, double &vb) {
  if (v16 && wa && wb) {
    const double2 v = *(const double2 *)(p + xa);
    va = v.x;
    vb = v.y;
  } else {
    va = wa ? p[xa] : 0.0;
    vb = wb ? p[xa + 1] : 0.0;
  }
}

template <bool FIX, int OP, bool INNER>
__device__ __forceinline__ void compute_plane2(const OpArgs &a, int64_t z, int x0, int y0, int R,
                                               const long long *lo, const long long *ce, const long long *up,
                                               double &rr, double &ff) {
  const Geo &q = a.q;
  const int nx = (int)q.nx, ny = (int)q.ny, pitch = (int)q.pitch;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col = 2 * lane, r0 = 1 + 4 * warp;
  const int xa = x0 - 2 + col;  // >= x0 >= 0 on output lanes
  const bool zin = z >= 1 && z < q.nz;
  const bool lane_out = lane >= 1 && lane <= 30;
  const bool oka = INNER || xa <= nx, okb = INNER || xa + 1 <= nx;
  const bool ina = INNER || (xa >= 1 && xa < nx), inb = INNER || (xa + 1 >= 1 && xa + 1 < nx);
  const double *fp = a.f ? a.f + z * q.plane : nullptr;
  const double *up_src = a.u + z * q.plane;
  double fa[4], fb[4], ua[4], ub[4];
  if (OP != OP_APPLY) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int j = y0 - 1 + r0 + k;
      const bool ok = lane_out && (INNER || j <= ny);
      const bool jin = ok && zin && (INNER || (j >= 1 && j < ny));
      ldg2(fp + j * pitch, xa, jin && ina, jin && inb, a.v16, fa[k], fb[k]);
      if (OP == OP_JACOBI)
        ldg2(up_src + j * pitch, xa, ok && oka, ok && okb, a.v16, ua[k], ub[k]);
    }
  }
  const int e2 = R - fx::FRAC;
  constexpr bool CVT = OPS3_CVT[OP], CVTB = CVT && !OPS3_SPLIT[OP];
  const double cf = OP == OP_JACOBI ? a.c2 : a.c1;
  const double sc = FIX && CVT ? cf * fx::pow2d(e2) : cf;
  const double scb = FIX && CVTB ? sc : (FIX ? cf : sc);  // the odd column's factor
  auto conv = [&](long long T, bool cvt) -> double { return cvt ? __ll2double_rn(T) : fx::to_double(T, e2); };
  const long long *lc = lo + col, *uc = up + col, *cc = ce + col;
  LL2 Cm = lds2(cc + (r0 - 1) * OS_W), Cc = lds2(cc + r0 * OS_W);
  LL2 Wm = add2<FIX>(lds2(lc + (r0 - 1) * OS_W), lds2(uc + (r0 - 1) * OS_W));
  LL2 Wc = add2<FIX>(lds2(lc + r0 * OS_W), lds2(uc + r0 * OS_W));
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = r0 + k;
    const LL2 Cp = lds2(cc + (r + 1) * OS_W);
    const LL2 Wp = add2<FIX>(lds2(lc + (r + 1) * OS_W), lds2(uc + (r + 1) * OS_W));
    const LL2 V = add2<FIX>(Cm, Cp);
    const LL2 Q = add2<FIX>(Wm, Wp);
    const LL2 VW = add2<FIX>(V, Wc);
    const LL2 P = add2<FIX>(add2<FIX>(VW, VW), Q);
    const long long Pl = __shfl_up_sync(0xffffffffu, P.b, 1);
    const long long Pr = __shfl_down_sync(0xffffffffu, P.a, 1);
    const LL2 Cu = Cc;
    Cm = Cc;
    Cc = Cp;
    Wm = Wc;
    Wc = Wp;
    const int j = y0 - 1 + r;
    if (!INNER && j > ny) continue;  // warp-uniform
    const bool jin = zin && (INNER || (j >= 1 && j < ny));
    // every lane computes (no branch around the halo lanes); only output lanes store
    const bool ia = jin && ina && lane_out, ib = jin && inb && lane_out;
    // 12 S u = 32 u - (2E + C); Td * sc is its term
    double Ta = 0.0, Tb = 0.0;
    {
      const long long Sa = add<FIX>(add<FIX>(Pl, P.b), add<FIX>(Q.a, Q.a));
      const long long Sb = add<FIX>(add<FIX>(P.a, Pr), add<FIX>(Q.b, Q.b));
      if (FIX) {
        Ta = conv(32 * Cu.a - Sa, CVT);
        Tb = conv(32 * Cu.b - Sb, CVTB);
      } else {
        Ta = fma(32.0, __longlong_as_double(Cu.a), -__longlong_as_double(Sa));
        Tb = fma(32.0, __longlong_as_double(Cu.b), -__longlong_as_double(Sb));
      }
    }
    const int off = j * pitch + xa;
    double oa, ob;
    if (OP == OP_APPLY) {
      oa = ia ? Ta * sc : 0.0;
      ob = ib ? Tb * scb : 0.0;
    } else if (OP == OP_JACOBI) {
      oa = ia ? fma(sc, Ta, fma(a.c1, fa[k], ua[k])) : ua[k];
      ob = ib ? fma(scb, Tb, fma(a.c1, fb[k], ub[k])) : ub[k];
    } else {
      oa = ia ? fma(sc, Ta, fa[k]) : 0.0;
      ob = ib ? fma(scb, Tb, fb[k]) : 0.0;
      if (ia) {
        rr = fma(oa, oa, rr);
        ff = fma(fa[k], fa[k], ff);
      }
      if (ib) {
        rr = fma(ob, ob, rr);
        ff = fma(fb[k], fb[k], ff);
      }
    }
    if (OP == OP_RESIDUAL && (!a.out || a.out_kind != 0)) {
      if (a.out) {
        const int64_t e = z * q.plane + off;  // element index
        if (a.out_kind == 1) {
          if (lane_out && oka) ((float *)a.out)[e] = (float)oa;
          if (lane_out && okb) ((float *)a.out)[e + 1] = (float)ob;
        } else {
          if (lane_out && oka) ((__nv_bfloat16 *)a.out)[e] = __float2bfloat16_rn((float)oa);
          if (lane_out && okb) ((__nv_bfloat16 *)a.out)[e + 1] = __float2bfloat16_rn((float)ob);
        }
      }
      continue;
    }
    double *op = a.out + z * q.plane + off;
    if (a.v16 && lane_out && oka && okb) {
      *(double2 *)op = make_double2(oa, ob);
    } else {
      if (lane_out && oka) op[0] = oa;
      if (lane_out && okb) op[1] = ob;
    }
  }
}

// Residual norms: fixed-order CTA sum, one partial per CTA, the last CTA adds the
// partials in order (deterministic for a given grid).
__device__ __forceinline__ void ops3_reduce_norms(const OpArgs &a, double rr, double ff, double *sh2, bool *last_p) {
  bool &last = *last_p;
  // fixed-order CTA sum, one partial per CTA, the last CTA adds them in order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
    ff += __shfl_xor_sync(0xffffffffu, ff, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sh2[2 * w] = rr;
    sh2[2 * w + 1] = ff;
  }
  __syncthreads();
  const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
  const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int k = 0; k < O_THREADS / 32; ++k) {
      s0 += sh2[2 * k];
      s1 += sh2[2 * k + 1];
    }
    a.partials[2 * bid] = s0;
    a.partials[2 * bid + 1] = s1;
    __threadfence();
    last = atomicAdd(a.counter, 1u) == nblk - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s0 = 0.0, s1 = 0.0;
  for (unsigned k = threadIdx.x; k < nblk; k += O_THREADS) {
    s0 += __ldcg(a.partials + 2 * k);
    s1 += __ldcg(a.partials + 2 * k + 1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  __syncthreads();
  if (l == 0) {
    sh2[2 * w] = s0;
    sh2[2 * w + 1] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int k = 0; k < O_THREADS / 32; ++k) {
      t0 += sh2[2 * k];
      t1 += sh2[2 * k + 1];
    }
    a.norms2[0] = t0;
    a.norms2[1] = t1;
    *a.counter = 0u;
  }
}

// CTAs per SM the register allocation targets: 3 (at most 85 registers) for the apply
// and the residual; the Jacobi sweep keeps more values live and runs faster at 2.
template <int OP>
constexpr int ops3_min_blocks() { return OP == OP_JACOBI ? 2 : 3; }

template <int OP>
__global__ void __launch_bounds__(O_THREADS, ops3_min_blocks<OP>()) k_ops3(OpArgs a) {
  extern __shared__ long long smem[];
  __shared__ int red[O_THREADS / 32];
  __shared__ double sh2[2 * O_THREADS / 32];
  __shared__ bool last;
  const Geo &q = a.q;
  const int64_t x0 = (int64_t)blockIdx.x * OT_X, y0 = (int64_t)blockIdx.y * OT_Y;
  const int64_t zs = (int64_t)blockIdx.z * a.cz;
  const int64_t ze = zs + a.cz < q.nz + 1 ? zs + a.cz : q.nz + 1;
  auto slot = [&](int i) -> long long * { return smem + i * (OS_H * OS_W); };
  // interior tile: every staged vertex in the grid, every output an interior vertex
  const bool inner_tile = x0 >= 1 && x0 + OT_X <= q.nx && y0 >= 1 && y0 + OT_Y <= q.ny;
  int lo = 0, ce = 1, up = 2;
  bool fix = true;
  int R = R_MIN;  // grows only
  double rr = 0.0, ff = 0.0;
  double v[O_PER];

  // Admit one prefetched plane into slot `dst`: agree on the scale, rescale or switch
  // to FP64 if needed, then store.  `live` slots hold already staged planes.
  auto admit = [&](int dst, int live0, int live1) {
    const int em = cta_max_exponent(v, red);
    if (fix && em != 0) {
      const int Rp = em - 1022 + 1;  // one spare bit
      const int Rn = Rp > R ? Rp : R;
      if (em == 2047 || Rp > R_MAX || Rp < R_MIN) {
        // Out of the fixed-point range (or all data seen so far below it): continue in
        // FP64.  Rp < R_MIN with R == R_MIN means nothing larger has been seen.
        if (em == 2047 || Rp > R_MAX || R == R_MIN) {
          for (int idx = threadIdx.x; idx < OS_H * OS_W; idx += O_THREADS) {
            slot(live0)[idx] = __double_as_longlong(fx::to_double(slot(live0)[idx], R - fx::FRAC));
            slot(live1)[idx] = __double_as_longlong(fx::to_double(slot(live1)[idx], R - fx::FRAC));
          }
          fix = false;
        }
      } else if (Rn > R) {
        const int d = Rn - R;
        for (int idx = threadIdx.x; idx < OS_H * OS_W; idx += O_THREADS) {
          slot(live0)[idx] = d < 63 ? (slot(live0)[idx] >> d) : (slot(live0)[idx] >> 63);
          slot(live1)[idx] = d < 63 ? (slot(live1)[idx] >> d) : (slot(live1)[idx] >> 63);
        }
        R = Rn;
      }
    }
    __syncthreads();  // red[] reuse, rescaled slots visible
#pragma unroll
    for (int k = 0; k < O_PER; ++k) {
      const int idx = threadIdx.x + k * O_THREADS;
      if (idx < OS_H * OS_W)
        slot(dst)[idx] = fix ? fx::to_fixed(v[k], 1023 + R) : __double_as_longlong(v[k]);
    }
  };

  // prologue: planes zs-1 and zs
  for (int idx = threadIdx.x; idx < 3 * OS_H * OS_W; idx += O_THREADS) smem[idx] = 0;
  __syncthreads();
  prefetch_plane(v, q, a.u, zs - 1, x0, y0);
  admit(lo, ce, up);
  prefetch_plane(v, q, a.u, zs, x0, y0);
  admit(ce, lo, up);
  prefetch_plane(v, q, a.u, zs + 1, x0, y0);
  for (int64_t z = zs; z < ze; ++z) {
    admit(up, lo, ce);
    __syncthreads();
    if (z + 2 <= ze) prefetch_plane(v, q, a.u, z + 2, x0, y0);
    if (fix) {
      if (inner_tile)
        compute_plane<true, OP, true>(a, z, (int)x0, (int)y0, R, slot(lo), slot(ce), slot(up), rr, ff);
      else
        compute_plane<true, OP, false>(a, z, (int)x0, (int)y0, R, slot(lo), slot(ce), slot(up), rr, ff);
    } else {
      compute_plane<false, OP, false>(a, z, (int)x0, (int)y0, R, slot(lo), slot(ce), slot(up), rr, ff);
    }
    __syncthreads();
    const int t = lo;
    lo = ce;
    ce = up;
    up = t;
  }

  if (OP == OP_RESIDUAL) ops3_reduce_norms(a, rr, ff, sh2, &last);
}

// ------------------------------------------------------------ TMA-staged form
// Same computation as k_ops3, with the planes brought into shared memory by TMA: four
// plane slots (lo, ce, up and the plane two ahead, which is in flight while the
// current plane computes), one mbarrier each.  The staged box starts at x0 - 2 (an even
// x, as TMA requires), so staged column c is x0 - 2 + c; the lanes work on column
// pairs (compute_plane2) or, reading the box one column to the right, on single columns
// as in k_ops3 (compute_plane).  A plane arrives as FP64 bits and is converted in place
// after the CTA agreed on the scale.  Wait limits: a TMA wait that runs out sets
// g_ops3_tma_error and the CTA leaves.
__device__ unsigned g_ops3_tma_error = 0;
constexpr unsigned OT_WAIT_LIMIT = 1u << 22;
constexpr unsigned OT_BOX_BYTES = OS_H * OS_W * 8;

template <int OP>
__global__ void __launch_bounds__(O_THREADS, ops3_min_blocks<OP>())
    k_ops3t(OpArgs a, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ int red[O_THREADS / 32];
  __shared__ double sh2[2 * O_THREADS / 32];
  __shared__ __align__(8) uint64_t bars[4];
  __shared__ bool last;
  __shared__ int fail;
  long long *smem = (long long *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  const Geo &q = a.q;
  const int64_t x0 = (int64_t)blockIdx.x * OT_X, y0 = (int64_t)blockIdx.y * OT_Y;
  const int64_t zs = (int64_t)blockIdx.z * a.cz;
  const int64_t ze = zs + a.cz < q.nz + 1 ? zs + a.cz : q.nz + 1;
  auto slot = [&](int i) -> long long * { return smem + i * (OS_H * OS_W); };
  const bool inner_tile = x0 >= 1 && x0 + OT_X <= q.nx && y0 >= 1 && y0 + OT_Y <= q.ny;
  int lo = 0, ce = 1, up = 2, nx = 3;
  unsigned phase = 0;  // bit i: parity of the next completion on slot i
  unsigned pend = 0;   // bit i: a load into slot i not yet waited for
  bool fix = true;
  int R = R_MIN;
  double rr = 0.0, ff = 0.0;
  double v[O_PER];
  if (threadIdx.x == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(&bars[i], 1);
    fail = 0;
    fence_mbar_init();
    fence_proxy_async();
  }
  __syncthreads();
  auto issue = [&](int s, int64_t z) {
    pend |= 1u << s;
    if (threadIdx.x == 0) {
      fence_proxy_async();  // earlier generic accesses to this slot before the TMA writes it
      tma_load_plane(slot(s), &tmap, (int)(x0 - 2), (int)(y0 - 1), (int)z, &bars[s], OT_BOX_BYTES);
    }
  };
  // Wait for slot dst, agree on the scale (rescaling the live slots if it grows), then
  // convert the slot in place.  Live slots are the already converted ones (-1: none);
  // a slot with a load in flight is never touched.  Returns false if the wait ran out.
  auto admit = [&](int dst, int live0, int live1) -> bool {
    if (mbar_wait(&bars[dst], (phase >> dst) & 1u, OT_WAIT_LIMIT)) {
      phase ^= 1u << dst;
      pend &= ~(1u << dst);
    } else {
      atomicExch(&fail, 1);  // the load stays pending
    }
#pragma unroll
    for (int k = 0; k < O_PER; ++k) {
      const int idx = threadIdx.x + k * O_THREADS;
      v[k] = idx < OS_H * OS_W ? __longlong_as_double(slot(dst)[idx]) : 0.0;
    }
    const int em = cta_max_exponent(v, red);  // includes a barrier
    if (fail) return false;
    if (fix && em != 0) {
      const int Rp = em - 1022 + 1;
      const int Rn = Rp > R ? Rp : R;
      if (em == 2047 || Rp > R_MAX || Rp < R_MIN) {
        if (em == 2047 || Rp > R_MAX || R == R_MIN) {
          for (int idx = threadIdx.x; idx < OS_H * OS_W; idx += O_THREADS) {
            if (live0 >= 0) slot(live0)[idx] = __double_as_longlong(fx::to_double(slot(live0)[idx], R - fx::FRAC));
            if (live1 >= 0) slot(live1)[idx] = __double_as_longlong(fx::to_double(slot(live1)[idx], R - fx::FRAC));
          }
          fix = false;
        }
      } else if (Rn > R) {
        const int d = Rn - R;
        for (int idx = threadIdx.x; idx < OS_H * OS_W; idx += O_THREADS) {
          if (live0 >= 0) slot(live0)[idx] = d < 63 ? (slot(live0)[idx] >> d) : (slot(live0)[idx] >> 63);
          if (live1 >= 0) slot(live1)[idx] = d < 63 ? (slot(live1)[idx] >> d) : (slot(live1)[idx] >> 63);
        }
        R = Rn;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < O_PER; ++k) {
      const int idx = threadIdx.x + k * O_THREADS;
      if (idx < OS_H * OS_W) slot(dst)[idx] = fix ? fx::to_fixed(v[k], 1023 + R) : __double_as_longlong(v[k]);
    }
    return true;
  };

  issue(lo, zs - 1);
  issue(ce, zs);
  issue(up, zs + 1);
  bool ok = admit(lo, -1, -1) && admit(ce, lo, -1);
  for (int64_t z = zs; z < ze && ok; ++z) {
    ok = admit(up, lo, ce);
    __syncthreads();
    if (!ok) break;
    if (z + 2 <= ze) issue(nx, z + 2);
    constexpr bool PAIRS = OPS3_PAIRS[OP];
    if (PAIRS) {
      if (fix) {
        if (inner_tile)
          compute_plane2<true, OP, true>(a, z, (int)x0, (int)y0, R, slot(lo), slot(ce), slot(up), rr, ff);
        else
          compute_plane2<true, OP, false>(a, z, (int)x0, (int)y0, R, slot(lo), slot(ce), slot(up), rr, ff);
      } else {
        compute_plane2<false, OP, false>(a, z, (int)x0, (int)y0, R, slot(lo), slot(ce), slot(up), rr, ff);
      }
    } else {
      // one column per lane: the staged box starts one column left of k_ops3's, so
      // read it shifted by one
      if (fix) {
        if (inner_tile)
          compute_plane<true, OP, true>(a, z, (int)x0, (int)y0, R, slot(lo) + 1, slot(ce) + 1, slot(up) + 1, rr,
                                        ff);
        else
          compute_plane<true, OP, false>(a, z, (int)x0, (int)y0, R, slot(lo) + 1, slot(ce) + 1, slot(up) + 1, rr,
                                         ff);
      } else {
        compute_plane<false, OP, false>(a, z, (int)x0, (int)y0, R, slot(lo) + 1, slot(ce) + 1, slot(up) + 1, rr,
                                        ff);
      }
    }
    __syncthreads();
    const int t = lo;
    lo = ce;
    ce = up;
    up = nx;
    nx = t;
  }
  // a wait ran out: the results are incomplete and the flag records it; every load
  // still in flight is waited for once more (bounded) so that none lands after the CTA
  // has left, and the CTA still takes part in the norm reduction so that its counter
  // stays consistent
  if (!ok) {
    for (int s = 0; s < 4; ++s)
      if (pend & (1u << s)) mbar_wait(&bars[s], (phase >> s) & 1u, OT_WAIT_LIMIT);
    if (threadIdx.x == 0) atomicExch(&g_ops3_tma_error, 1u);
  }
  if (OP == OP_RESIDUAL) ops3_reduce_norms(a, rr, ff, sh2, &last);
}

// Planes per CTA; the stencil apply may take a tuned value (the residual may not: its
// reduction workspace is sized from this grid).
int ops_cz(const Geo &q, bool tuned) {
  const int64_t txy = ((q.nx + OT_X) / OT_X) * ((q.ny + OT_Y) / OT_Y);
  const int cz = z_chunk(txy, q.nz + 1, O_CZ, 4, 3);
  return tuned ? tuned_chunk(tuning_lookup(STENCIL_CALL_APPLY_STENCIL, q), cz, 4, O_CZ) : cz;
}

dim3 ops_grid(const Geo &q, bool tuned) {
  const int cz = ops_cz(q, tuned);
  return dim3((unsigned)((q.nx + OT_X) / OT_X), (unsigned)((q.ny + OT_Y) / OT_Y),
              (unsigned)((q.nz + cz) / cz));
}

template <int OP>
cudaError_t launch_op(const OpArgs &a, cudaStream_t s) {
  static PerDeviceOnce attr;
  {
    cudaError_t e = set_smem_limit_once(attr, k_ops3<OP>, O_SMEM);
    if (e != cudaSuccess) return e;
  }
  const dim3 g = ops_grid(a.q, OP == OP_APPLY);
  if (g.y > 65535 || g.z > 65535) return cudaErrorInvalidConfiguration;
  if (a.q.plane >= ((int64_t)1 << 31) - OS_W * OS_H) return cudaErrorInvalidValue;
  OpArgs b = a;
  b.cz = ops_cz(a.q, OP == OP_APPLY);
  b.v16 = a.q.pitch % 2 == 0 && ((uintptr_t)a.f % 16) == 0 &&
          (a.out_kind != 0 || ((uintptr_t)a.out % 16) == 0);
  CUtensorMap map;
  if (tma_plane_map(a.q, a.u, OS_W, OS_H, &map)) {
    constexpr size_t smem_t = 4 * (size_t)OS_H * OS_W * sizeof(long long) + 128;
    static PerDeviceOnce attr_t;
    cudaError_t e = set_smem_limit_once(attr_t, k_ops3t<OP>, smem_t);
    if (e != cudaSuccess) return e;
    k_ops3t<OP><<<g, O_THREADS, smem_t, s>>>(b, map);
  } else {
    k_ops3<OP><<<g, O_THREADS, O_SMEM, s>>>(b);
  }
  return cudaGetLastError();
}


}  // namespace

size_t ops_fx_reduce_bytes(const Geo &q) {
  const dim3 g = ops_grid(q, false);
  return (size_t)g.x * g.y * g.z * 2 * sizeof(double) + 16;
}

cudaError_t launch_apply_stencil_fx3(const Geo &q, const double *u, double *y, cudaStream_t s) {
  OpArgs a{};
  a.q = q;
  a.u = u;
  a.out = y;
  a.c1 = 1.0 / (12.0 * q.h * q.h);
  return launch_op<OP_APPLY>(a, s);
}

cudaError_t launch_jacobi_fx3(const Geo &q, const double *u, const double *f, double *unew,
                              double omega, cudaStream_t s) {
  OpArgs a{};
  a.q = q;
  a.u = u;
  a.f = f;
  a.out = unew;
  a.c1 = omega * 0.375 * q.h * q.h;
  a.c2 = -omega * 0.375 / 12.0;
  return launch_op<OP_JACOBI>(a, s);
}

cudaError_t launch_residual_fx3(const Geo &q, const double *u, const double *f, double *r,
                                double *norms2, void *scratch, cudaStream_t s, int out_kind) {
  OpArgs a{};
  a.q = q;
  a.u = u;
  a.f = f;
  a.out = r;
  a.c1 = -1.0 / (12.0 * q.h * q.h);
  a.counter = (unsigned *)scratch;  // counter first, partials after (same layout everywhere)
  a.partials = (double *)((char *)scratch + 16);
  a.norms2 = norms2;
  a.out_kind = out_kind;
  return launch_op<OP_RESIDUAL>(a, s);
}

}  // namespace stencil

namespace stencil {

// The TMA wait flag of this file's kernels (1 once a bounded wait ran out); cleared on
// request.  Synchronous.
cudaError_t tma_wait_flag_ops3(unsigned *value, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(value, g_ops3_tma_error, sizeof(unsigned));
  if (e == cudaSuccess && clear && *value) {
    const unsigned zero = 0u;
    e = cudaMemcpyToSymbol(g_ops3_tma_error, &zero, sizeof(unsigned));
  }
  return e;
}

}  // namespace stencil
