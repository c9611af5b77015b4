// 2D Q1 (bilinear, 9-point stencil of Fig. 1) operations on the integer pipes:
// assembled apply, element-wise apply with colour passes, damped Jacobi sweep,
// residual with norms, and the coloured Gauss-Seidel sweep (one pass per sweep).
//
//   3 S u = 8 u - N,  N = sum of the 8 neighbours;   6 K_e (element matrix, h-free) has
//   entries 4 (same vertex), -1 (differ in one coordinate), -2 (opposite corner).
// Values are int64 fixed point (fixed.cuh); N is formed from column sums
//   V = u(j-1) + u(j+1),  T = V + u(j),  N(x) = T(x-1) + T(x+1) + V(x).
//
// Each warp owns a segment of 32 consecutive columns and streams down a chunk of rows,
// keeping the rows it needs in registers and reaching x-neighbours by shuffles; no
// shared memory and no block barriers.  For the single-pass operations the fixed-point
// reference R is per warp and only grows: every newly loaded row is reduced to its
// largest exponent first, and when that exceeds R the rows held so far are shifted to
// the new scale.  A warp that meets
// a non-finite value or magnitudes outside [2^-900, 2^1000] converts what it holds to
// FP64 and continues in native FP64 arithmetic.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fixed.cuh"
#include "internal.h"
#include "sweep_bounds.cuh"

namespace stencil {
namespace {

constexpr int W2_THREADS = 128;
constexpr int W2_ROWS = 64;   // rows per warp (single-pass operations)
constexpr int S2_ROWS = 256;  // rows per warp (multi-sweep GS and Jacobi)
constexpr int R_MIN = -900, R_MAX = 1000;

enum { O2_APPLY = 0, O2_JACOBI = 1, O2_RESIDUAL = 2, O2_ELEMENTWISE = 3 };

struct Op2Args {
  Geo q;
  const double *u, *f;
  double *out;
  double c1, c2;
  double *partials;
  unsigned *counter;
  double *norms2;
};

struct WarpScale {
  bool fix = true;
  int R = R_MIN;
};

__device__ __forceinline__ unsigned biased_exp(double v) {
  return (unsigned)(fx::dbits(v) >> 52) & 0x7ffu;
}

// Agree on the scale for a new row whose largest biased exponent over the warp is em
// (headroom: extra spare bits).  Returns the right shift to apply to values already
// held (0 if none), or -1 when the warp must switch to FP64.
__device__ __forceinline__ int admit_row(WarpScale &w, unsigned em, int headroom) {
  if (!w.fix || em == 0) return 0;
  const int Rp = (int)em - 1022 + headroom;
  if (em == 2047 || Rp > R_MAX || (Rp < R_MIN && w.R == R_MIN)) return -1;
  if (Rp > w.R) {
    const int d = Rp - w.R;
    w.R = Rp;
    return d;
  }
  return 0;
}

__device__ __forceinline__ long long shr(long long v, int d) { return d >= 63 ? (v >> 63) : (v >> d); }

__device__ __forceinline__ long long to_f64_bits(long long v, int R) {
  return __double_as_longlong(fx::to_double(v, R - fx::FRAC));
}

template <bool FIX>
__device__ __forceinline__ long long add(long long a, long long b) {
  if (FIX) return a + b;
  return __double_as_longlong(__longlong_as_double(a) + __longlong_as_double(b));
}

// 8u - N at this lane's column (3 S u), from the rows above (m), at (c) and below (p).
template <bool FIX>
__device__ __forceinline__ long long eight_u_minus_n(long long m, long long c, long long p) {
  const long long V = add<FIX>(m, p);
  const long long T = add<FIX>(V, c);
  const long long Tm = __shfl_up_sync(0xffffffffu, T, 1);
  const long long Tp = __shfl_down_sync(0xffffffffu, T, 1);
  const long long N = add<FIX>(add<FIX>(Tm, Tp), V);
  if (FIX) return 8 * c - N;
  return __double_as_longlong(fma(8.0, __longlong_as_double(c), -__longlong_as_double(N)));
}

constexpr int PF = 3;  // rows in flight per warp

// Per-warp streaming state of k_ops2.
struct Stream2 {
  int64_t x;
  bool xok, xin, out_lane;
  int lane;
  long long um, uc, up;  // converted rows j-1, j, j+1 (element-wise: ua = uc, acc = um/up)
  double rc, rp;         // raw rows j, j+1
  double rr, ff;
};

// Element-wise apply: cell rows cj in [cj0, je); returns the first row not done (a
// switch to FP64 was requested) or je.
template <bool FIX>
__device__ __forceinline__ int64_t ew2_rows(const Op2Args &a, WarpScale &w, Stream2 &s, int64_t cj0, int64_t js,
                                            int64_t je) {
  const Geo &q = a.q;
  const double *ucol = a.u + (s.xok ? s.x : 0);
  long long &ua = s.uc, &alo = s.um, &ahi = s.up;
  double qb[PF];  // qb[t]: raw vertex row cj + 1 for the iteration cj = cb + t
#pragma unroll
  for (int t = 0; t < PF; ++t)
    qb[t] = (s.xok && cj0 + 1 + t <= q.ny && cj0 + 1 + t >= 0) ? ucol[(cj0 + 1 + t) * q.pitch] : 0.0;
  for (int64_t cb = cj0; cb < je; cb += PF) {
#pragma unroll
    for (int t = 0; t < PF; ++t) {
      const int64_t cj = cb + t;
      if (cj >= je) return je;
      const int slot = t;
      const double rb = qb[slot];
      const unsigned em = __reduce_max_sync(0xffffffffu, biased_exp(rb));
      if (FIX) {
        const int d = admit_row(w, em, 1);
        if (d < 0) {  // leave this row to the FP64 loop
          ua = to_f64_bits(ua, w.R);
          alo = to_f64_bits(alo, w.R);
          ahi = to_f64_bits(ahi, w.R);
          w.fix = false;
          return cj;
        }
        if (d > 0) {
          ua = shr(ua, d);
          alo = shr(alo, d);
          ahi = shr(ahi, d);
        }
      }
      qb[slot] = (cj + 1 + PF <= je && s.xok && cj + 1 + PF <= q.ny) ? ucol[(cj + 1 + PF) * q.pitch] : 0.0;
      const long long ub = FIX ? fx::to_fixed(rb, 1023 + w.R) : __double_as_longlong(rb);
      // cell with lower-left vertex (x, cj): v0 = (x,cj), v1 = (x+1,cj), v2 = (x,cj+1),
      // v3 = (x+1,cj+1); 6 (K u)_w = 4 u_w - (face-adjacent pair) - 2 u_opposite
      const long long v1 = __shfl_down_sync(0xffffffffu, ua, 1);
      const long long v3 = __shfl_down_sync(0xffffffffu, ub, 1);
      const bool cell = s.lane <= 30 && s.x >= 0 && s.x < q.nx && cj >= 0 && cj < q.ny;
      // Every lane forms its own cell's four contributions; each vertex column is owned
      // by one lane, which adds the share of its own cell and (by shuffle) that of the
      // cell on its left, so the scatter has no write conflicts.  In fixed point the
      // sums are exact, so the order of the two x colours is immaterial; the FP64 path
      // adds the even-x colour's share first.
      long long c0 = 0, c1 = 0, c2 = 0, c3 = 0;
      if (cell) {
        if (FIX) {
          const long long s1 = v1 + ub, s2 = ua + v3;
          c0 = 4 * ua - s1 - 2 * v3;
          c1 = 4 * v1 - s2 - 2 * ub;
          c2 = 4 * ub - s2 - 2 * v1;
          c3 = 4 * v3 - s1 - 2 * ua;
        } else {
          const double A0 = __longlong_as_double(ua), A1 = __longlong_as_double(v1),
                       A2 = __longlong_as_double(ub), A3 = __longlong_as_double(v3);
          c0 = __double_as_longlong(4.0 * A0 - (A1 + A2) - 2.0 * A3);
          c1 = __double_as_longlong(4.0 * A1 - (A0 + A3) - 2.0 * A2);
          c2 = __double_as_longlong(4.0 * A2 - (A0 + A3) - 2.0 * A1);
          c3 = __double_as_longlong(4.0 * A3 - (A1 + A2) - 2.0 * A0);
        }
      }
      long long c1l = __shfl_up_sync(0xffffffffu, c1, 1), c3l = __shfl_up_sync(0xffffffffu, c3, 1);
      if (s.lane == 0) c1l = c3l = 0;
      if (FIX || (s.x & 1) == 0) {  // own cell has the even-x colour: it goes first
        alo = add<FIX>(add<FIX>(alo, c0), c1l);
        ahi = add<FIX>(add<FIX>(ahi, c2), c3l);
      } else {
        alo = add<FIX>(add<FIX>(alo, c1l), c0);
        ahi = add<FIX>(add<FIX>(ahi, c3l), c2);
      }
      if (cj >= js && s.out_lane) {
        const bool inner = s.xin && cj >= 1 && cj < q.ny;
        // FIX: 2^(R-52) c1 times the converted sum (exact power-of-two scaling of c1)
        const double sv = FIX ? __ll2double_rn(alo) : __longlong_as_double(alo);
        a.out[cj * q.pitch + s.x] = inner ? sv * (FIX ? a.c1 * fx::pow2d(w.R - fx::FRAC) : a.c1) : 0.0;
      }
      alo = ahi;
      ahi = 0;
      ua = ub;
    }
  }
  return je;
}

// Assembled apply / Jacobi / residual: output rows j in [j0, je).
template <bool FIX, int OP>
__device__ __forceinline__ int64_t op2_rows(const Op2Args &a, WarpScale &w, Stream2 &s, int64_t j0, int64_t js,
                                            int64_t je) {
  const Geo &q = a.q;
  const double *ucol = a.u + (s.xok ? s.x : 0);
  const double *fcol = a.f ? a.f + (s.xok ? s.x : 0) : nullptr;
  double *ocol = a.out ? a.out + (s.xok ? s.x : 0) : nullptr;
  double qb[PF];  // qb[t]: raw row j + 2 for the iteration j = jb + t
#pragma unroll
  for (int t = 0; t < PF; ++t) qb[t] = (s.xok && j0 + 2 + t <= q.ny) ? ucol[(j0 + 2 + t) * q.pitch] : 0.0;
  for (int64_t jb = j0; jb < je; jb += PF) {
#pragma unroll
    for (int t = 0; t < PF; ++t) {
      const int64_t j = jb + t;
      if (j >= je) return je;
      const int slot = t;
      const double rn = qb[slot];  // row j + 2
      const unsigned em = __reduce_max_sync(0xffffffffu, biased_exp(rn));
      const bool inner = s.xin && j >= 1 && j < q.ny;
      double fv = 0.0;
      if (OP != O2_APPLY && s.out_lane && inner) fv = fcol[j * q.pitch];
      const long long T = eight_u_minus_n<FIX>(s.um, s.uc, s.up);
      if (s.out_lane) {
        // converted on the integer pipe here (measured faster than the FP64 pipe's
        // conversion for these three operations; the element-wise apply uses the latter)
        const double Td = inner ? (FIX ? fx::to_double(T, w.R - fx::FRAC) : __longlong_as_double(T)) : 0.0;
        const int64_t go = j * q.pitch;
        if (OP == O2_APPLY) {
          ocol[go] = inner ? Td * a.c1 : 0.0;
        } else if (OP == O2_JACOBI) {
          ocol[go] = inner ? fma(a.c2, Td, fma(a.c1, fv, s.rc)) : s.rc;
        } else {
          const double r = inner ? fma(a.c1, Td, fv) : 0.0;
          if (ocol) ocol[go] = r;
          if (inner) {
            s.rr = fma(r, r, s.rr);
            s.ff = fma(fv, fv, s.ff);
          }
        }
      }
      // admit row j + 2 (after row j is done)
      if (FIX) {
        const int d = admit_row(w, em, 1);
        if (d < 0) {
          s.uc = to_f64_bits(s.uc, w.R);
          s.up = to_f64_bits(s.up, w.R);
          w.fix = false;
          // row j is finished; rows j+1, j+2 continue in FP64 (rn still in the queue)
          s.um = s.uc;
          s.uc = s.up;
          s.up = __double_as_longlong(rn);
          s.rc = s.rp;
          s.rp = rn;
          return j + 1;
        }
        if (d > 0) {
          s.uc = shr(s.uc, d);
          s.up = shr(s.up, d);
        }
      }
      qb[slot] = (j + 2 + PF <= je && s.xok && j + 2 + PF <= q.ny) ? ucol[(j + 2 + PF) * q.pitch] : 0.0;
      s.um = s.uc;
      s.uc = s.up;
      s.up = FIX ? fx::to_fixed(rn, 1023 + w.R) : __double_as_longlong(rn);
      s.rc = s.rp;
      s.rp = rn;
    }
  }
  return je;
}

// One warp's share of k_ops2: a segment of 30 output columns and a chunk of rows.
template <int OP>
__device__ __forceinline__ void ops2_warp(const Op2Args &a, int lane, int64_t gw, Stream2 &s, int rows) {
  const Geo &q = a.q;
  const int64_t nseg = (q.nx + 30) / 30;  // 30 outputs per segment
  const int64_t seg = gw % nseg, chunk = gw / nseg;
  const int64_t js = chunk * rows;
  const int64_t je = js + rows < q.ny + 1 ? js + rows : q.ny + 1;
  s.lane = lane;
  s.x = seg * 30 + lane - 1;  // lanes 1..30 produce outputs
  s.xok = s.x >= 0 && s.x <= q.nx;
  s.xin = s.x >= 1 && s.x < q.nx;
  s.out_lane = lane >= 1 && lane <= 30 && s.xok;
  s.rr = 0.0;
  s.ff = 0.0;
  WarpScale w;
  if (js <= q.ny) {
    const double *ucol = a.u + (s.xok ? s.x : 0);
    auto load = [&](int64_t j) -> double { return (s.xok && j >= 0 && j <= q.ny) ? ucol[j * q.pitch] : 0.0; };
    if (OP == O2_ELEMENTWISE) {
      const double ra = load(js - 1);
      if (admit_row(w, __reduce_max_sync(0xffffffffu, biased_exp(ra)), 1) < 0) w.fix = false;
      s.uc = w.fix ? fx::to_fixed(ra, 1023 + w.R) : __double_as_longlong(ra);
      s.um = 0;
      s.up = 0;
      int64_t cj = js - 1;
      if (w.fix) cj = ew2_rows<true>(a, w, s, cj, js, je);
      if (cj < je) ew2_rows<false>(a, w, s, cj, js, je);
    } else {
      s.rc = load(js);
      s.rp = load(js + 1);
      const double rm = load(js - 1);
      unsigned em = __reduce_max_sync(0xffffffffu, biased_exp(rm));
      em = max(em, __reduce_max_sync(0xffffffffu, biased_exp(s.rc)));
      em = max(em, __reduce_max_sync(0xffffffffu, biased_exp(s.rp)));
      if (admit_row(w, em, 1) < 0) w.fix = false;
      s.um = w.fix ? fx::to_fixed(rm, 1023 + w.R) : __double_as_longlong(rm);
      s.uc = w.fix ? fx::to_fixed(s.rc, 1023 + w.R) : __double_as_longlong(s.rc);
      s.up = w.fix ? fx::to_fixed(s.rp, 1023 + w.R) : __double_as_longlong(s.rp);
      int64_t j = js;
      if (w.fix) j = op2_rows<true, OP>(a, w, s, j, js, je);
      if (j < je) op2_rows<false, OP>(a, w, s, j, js, je);
    }
  }
}

template <int OP>
__global__ void __launch_bounds__(W2_THREADS) k_ops2(Op2Args a) {
  __shared__ double sh[2 * W2_THREADS / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  Stream2 s;
  ops2_warp<OP>(a, lane, (int64_t)blockIdx.x * (W2_THREADS / 32) + wib, s, W2_ROWS);
  double rr = s.rr, ff = s.ff;
  if (OP == O2_RESIDUAL) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rr += __shfl_xor_sync(0xffffffffu, rr, o);
      ff += __shfl_xor_sync(0xffffffffu, ff, o);
    }
    if (lane == 0) {
      sh[2 * wib] = rr;
      sh[2 * wib + 1] = ff;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s0 = 0.0, s1 = 0.0;
      for (int k = 0; k < W2_THREADS / 32; ++k) {
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
    for (unsigned k = threadIdx.x; k < gridDim.x; k += W2_THREADS) {
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
      sh[2 * wib] = s0;
      sh[2 * wib + 1] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double t0 = 0.0, t1 = 0.0;
      for (int k = 0; k < W2_THREADS / 32; ++k) {
        t0 += sh[2 * k];
        t1 += sh[2 * k + 1];
      }
      a.norms2[0] = t0;
      a.norms2[1] = t1;
      *a.counter = 0u;
    }
  }
}

unsigned ops2_blocks(const Geo &q) {
  const int64_t nseg = (q.nx + 30) / 30;
  const int64_t nchunk = (q.ny + W2_ROWS) / W2_ROWS;
  return (unsigned)((nseg * nchunk + W2_THREADS / 32 - 1) / (W2_THREADS / 32));
}

// ------------------------------------------------------------------ Gauss-Seidel
// u_new = 3/8 h^2 f + N/8.
// Whole sweep in one pass (row wavefront inside a warp).  For even row j: colours 0
// (x even) and 1 (x odd) from the old rows j-1, j+1; then odd row j-1: colours 2 and 3
// from the new rows j-2 and j.  Every value read is the one the sequential colour
// order would read.  Lanes cover 32 columns; each colour step consumes one lane of
// halo, so lanes 4..27 produce outputs (24 per segment).  A chunk of rows [js, je]
// (js even) also recomputes its last even row je (which the next chunk owns) so that
// its last odd row can be finished; chunks are therefore independent.
struct Gs2Lane {
  int64_t x;
  bool xok, xin, out_lane;
  long long ev_new;  // converted new even row j-2
  long long od_old;  // converted old odd row j-1
  double od_raw;     // raw old odd row j-1 (for Dirichlet copies)
};

template <bool FIX>
__device__ __forceinline__ void colour_pair(long long &uc, long long V, double fv, double g, const WarpScale &w,
                                            bool xin, int64_t x, double &out0) {
#pragma unroll
  for (int px = 0; px < 2; ++px) {
    const long long T = add<FIX>(V, uc);
    const long long Tm = __shfl_up_sync(0xffffffffu, T, 1);
    const long long Tp = __shfl_down_sync(0xffffffffu, T, 1);
    if (xin && (int)(x & 1) == px) {
      const long long Nn = add<FIX>(add<FIX>(Tm, Tp), V);
      double un;
      if (FIX) {
        un = fma(g, fv, fx::to_double(Nn, w.R - fx::FRAC - 3));
        uc = fx::to_fixed(un, 1023 + w.R);
      } else {
        un = fma(__longlong_as_double(Nn), 0.125, g * fv);
        uc = __double_as_longlong(un);
      }
      out0 = un;
    }
  }
}

template <bool FIX>
__device__ __forceinline__ int64_t gs2f_rows(const Geo &q, const double *__restrict__ X, double *__restrict__ Y,
                                             const double *__restrict__ f, double g, WarpScale &w, Gs2Lane &L,
                                             int64_t j0, int64_t js, int64_t je) {
  auto ldx = [&](int64_t j) -> double { return (L.xok && j >= 0 && j <= q.ny) ? X[j * q.pitch + L.x] : 0.0; };
  auto ldf = [&](int64_t j) -> double {
    return (L.xin && j >= 1 && j < q.ny) ? f[j * q.pitch + L.x] : 0.0;
  };
  constexpr int PG = 2;
  double qe[PG], qo[PG], qfe[PG], qfo[PG];  // X rows j, j+1 and f rows j, j-1 for even j
#pragma unroll
  for (int t = 0; t < PG; ++t) {
    const int64_t j = j0 + 2 * t;
    qe[t] = ldx(j);
    qo[t] = ldx(j + 1);
    qfe[t] = ldf(j);
    qfo[t] = ldf(j - 1);
  }
  for (int64_t jb = j0; jb <= je; jb += 2 * PG) {
#pragma unroll
    for (int t = 0; t < PG; ++t) {
      const int64_t j = jb + 2 * t;
      if (j > je) return je + 2;
      const double rc = qe[t], rp = qo[t], fe = qfe[t], fo = qfo[t];
      if (FIX) {
        unsigned em = __reduce_max_sync(0xffffffffu, biased_exp(rc));
        em = max(em, __reduce_max_sync(0xffffffffu, biased_exp(rp)));
        const unsigned ef = max(__reduce_max_sync(0xffffffffu, biased_exp(fe)),
                                __reduce_max_sync(0xffffffffu, biased_exp(fo)));
        if (ef) em = max(em, (unsigned)max(1, (int)ef + (int)biased_exp(g) - 1023 + 1));
        const int d = admit_row(w, em, 2);
        if (d < 0) {
          L.ev_new = to_f64_bits(L.ev_new, w.R);
          L.od_old = to_f64_bits(L.od_old, w.R);
          w.fix = false;
          return j;  // redo from this even row in FP64
        }
        if (d > 0) {
          L.ev_new = shr(L.ev_new, d);
          L.od_old = shr(L.od_old, d);
        }
      }
      {
        const int64_t jn = j + 2 * PG;
        qe[t] = jn <= je ? ldx(jn) : 0.0;
        qo[t] = jn <= je ? ldx(jn + 1) : 0.0;
        qfe[t] = jn <= je ? ldf(jn) : 0.0;
        qfo[t] = jn <= je ? ldf(jn - 1) : 0.0;
      }
      // even row j: colours 0 and 1 from the old rows j-1 (od_old) and j+1
      long long ue = FIX ? fx::to_fixed(rc, 1023 + w.R) : __double_as_longlong(rc);
      const long long up_old = FIX ? fx::to_fixed(rp, 1023 + w.R) : __double_as_longlong(rp);
      double oute = rc;
      if (j >= 1 && j < q.ny) colour_pair<FIX>(ue, add<FIX>(L.od_old, up_old), fe, g, w, L.xin, L.x, oute);
      // odd row j-1: colours 2 and 3 from the new rows j-2 (ev_new) and j (ue)
      if (j - 1 >= js + 1) {
        long long uo = L.od_old;
        double outo = L.od_raw;
        if (j - 1 < q.ny) colour_pair<FIX>(uo, add<FIX>(L.ev_new, ue), fo, g, w, L.xin, L.x, outo);
        if (L.out_lane) Y[(j - 1) * q.pitch + L.x] = outo;
      }
      if (L.out_lane && (j < je || je == q.ny)) Y[j * q.pitch + L.x] = oute;
      L.ev_new = ue;
      L.od_old = up_old;
      L.od_raw = rp;
    }
  }
  return je + 2;
}

// One warp's share of a sweep on FP64 data with the per-warp adaptive scale.
__device__ __forceinline__ void gs2_fused_warp(const Geo &q, const double *__restrict__ X, double *__restrict__ Y,
                                               const double *__restrict__ f, double g, int64_t seg, int64_t js,
                                               int lane, int rows) {
  // last even row of the chunk (recomputed; the next chunk writes it) or the grid end
  int64_t je = js + rows;
  if (je > q.ny) je = (q.ny & 1) ? q.ny + 1 : q.ny;
  Gs2Lane L;
  L.x = seg * 24 + lane - 4;
  L.xok = L.x >= 0 && L.x <= q.nx;
  L.xin = L.x >= 1 && L.x < q.nx;
  L.out_lane = lane >= 4 && lane <= 27 && L.xok;
  WarpScale w;
  const double rm = (L.xok && js - 1 >= 0) ? X[(js - 1) * q.pitch + L.x] : 0.0;
  if (admit_row(w, __reduce_max_sync(0xffffffffu, biased_exp(rm)), 2) < 0) w.fix = false;
  L.od_old = w.fix ? fx::to_fixed(rm, 1023 + w.R) : __double_as_longlong(rm);
  L.od_raw = rm;
  L.ev_new = 0;
  int64_t j = js;
  if (w.fix) j = gs2f_rows<true>(q, X, Y, f, g, w, L, j, js, je);
  if (j <= je) gs2f_rows<false>(q, X, Y, f, g, w, L, j, js, je);
}

__global__ void __launch_bounds__(W2_THREADS) k_gs2_fused(Geo q, const double *__restrict__ X,
                                                          double *__restrict__ Y, const double *__restrict__ f,
                                                          double g) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * (W2_THREADS / 32) + wib;
  const int64_t nseg = (q.nx + 24) / 24;
  const int64_t seg = gw % nseg, chunk = gw / nseg;
  const int64_t js = chunk * S2_ROWS;  // even
  if (js > q.ny) return;
  gs2_fused_warp(q, X, Y, f, g, seg, js, lane, S2_ROWS);
}

// ------------------------------------------------------------------ multi-sweep form
// Intermediate sweeps of one call keep the iterate as int64 fixed point in HBM at a
// scale shared by the whole grid and tracked on the device (sweep_bounds.cuh), and
// 3/8 h^2 f is precomputed once per call as fixed point (GF).  A sweep is then integer
// arithmetic only: no conversion per element except on the first load from u and the
// last store into u.  Same row wavefront as above.
enum { SF_F64 = 0, SF_FXP = 1 };  // storage format: FP64, or int64 fixed point

__device__ __forceinline__ void colour_pair_gs(long long &uc, long long V, long long gv, bool xin, int64_t x) {
#pragma unroll
  for (int px = 0; px < 2; ++px) {
    const long long T = V + uc;
    const long long Tm = __shfl_up_sync(0xffffffffu, T, 1);
    const long long Tp = __shfl_down_sync(0xffffffffu, T, 1);
    if (xin && (int)(x & 1) == px) uc = gv + ((Tm + Tp + V) >> 3);  // 3/8 h^2 f + N / 8
  }
}

template <int XF, int YF>
__global__ void __launch_bounds__(W2_THREADS) k_gs2_sweep(Geo q, const void *__restrict__ X, void *__restrict__ Y,
                                                          const double *__restrict__ f,
                                                          const long long *__restrict__ GF, SweepBounds *bnd,
                                                          int sweep, int sweeps, double g, bool write_bnd) {
  __shared__ long long red[W2_THREADS / 32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * (W2_THREADS / 32) + wib;
  const int64_t nseg = (q.nx + 24) / 24;
  const int64_t seg = gw % nseg, chunk = gw / nseg;
  const int64_t js = chunk * S2_ROWS;  // even
  const Plan plan = make_plan(bnd, g, sweeps);
  if (!plan.fix) {
    // bound unusable for fixed point: every sweep of the call keeps FP64 buffers
    if (js <= q.ny) gs2_fused_warp(q, (const double *)X, (double *)Y, f, g, seg, js, lane, S2_ROWS);
    return;
  }
  const int R = sweep_R(bnd, sweep % 4, g);
  const int Rx = sweep > 0 ? sweep_R(bnd, (sweep + 3) % 4, g) : R;
  const int dx = XF == SF_FXP ? R - Rx : 0, df = R - plan.Rf, rb = 1023 + R;
  // shift amounts clamped once: inputs by dx (right, or left when the scale shrank),
  // GF by df >= 0 (a shift by 63 leaves 0 or -1: below one unit of the last place)
  const int dxr = dx > 0 ? (dx < 63 ? dx : 63) : 0, dxl = dx < 0 ? (-dx < 63 ? -dx : 63) : 0;
  const int dfr = df < 63 ? df : 63;
  if (blockIdx.x == 0 && threadIdx.x == 0) bnd->umax[(sweep + 2) % 4] = 0ull;
  long long vmax = 0;
  if (js <= q.ny) {
    int64_t je = js + S2_ROWS;
    if (je > q.ny) je = (q.ny & 1) ? q.ny + 1 : q.ny;
    const int64_t x = seg * 24 + lane - 4;
    const bool xok = x >= 0 && x <= q.nx, xin = x >= 1 && x < q.nx;
    const bool out_lane = lane >= 4 && lane <= 27 && xok;
    const long long *Xl = (const long long *)X;
    auto rawx = [&](int64_t j) -> long long { return (xok && j >= 0 && j <= q.ny) ? Xl[j * q.pitch + x] : 0ll; };
    auto rawg = [&](int64_t j) -> long long { return (xin && j >= 1 && j < q.ny) ? GF[j * q.pitch + x] : 0ll; };
    auto cvx = [&](long long raw) -> long long {
      return XF == SF_F64 ? fx::to_fixed(__longlong_as_double(raw), rb) : (raw >> dxr) << dxl;
    };
    auto put = [&](int64_t j, long long v) {
      if (!out_lane) return;
      const bool inner = xin && j >= 1 && j < q.ny;
      if (!inner && !write_bnd) return;
      if (YF == SF_FXP)
        ((long long *)Y)[j * q.pitch + x] = v;
      else
        ((double *)Y)[j * q.pitch + x] = fx::to_double_cvt(v, R - fx::FRAC);
      const long long a = v < 0 ? -v : v;
      vmax = a > vmax ? a : vmax;
    };
    long long od_old = cvx(rawx(js - 1)), ev_new = 0;
    constexpr int PG = 2;
    long long qe[PG], qo[PG], qge[PG], qgo[PG];  // raw X rows j, j+1 and GF rows j, j-1
#pragma unroll
    for (int t = 0; t < PG; ++t) {
      const int64_t j = js + 2 * t;
      const bool ok = j <= je;
      qe[t] = ok ? rawx(j) : 0ll;
      qo[t] = ok ? rawx(j + 1) : 0ll;
      qge[t] = ok ? rawg(j) : 0ll;
      qgo[t] = ok ? rawg(j - 1) : 0ll;
    }
    for (int64_t jb = js; jb <= je; jb += 2 * PG) {
#pragma unroll
      for (int t = 0; t < PG; ++t) {
        const int64_t j = jb + 2 * t;
        if (j > je) break;
        const long long rc = cvx(qe[t]), rp = cvx(qo[t]);
        const long long ge = qge[t] >> dfr, go = qgo[t] >> dfr;
        {
          const int64_t jn = j + 2 * PG;
          const bool ok = jn <= je;
          qe[t] = ok ? rawx(jn) : 0ll;
          qo[t] = ok ? rawx(jn + 1) : 0ll;
          qge[t] = ok ? rawg(jn) : 0ll;
          qgo[t] = ok ? rawg(jn - 1) : 0ll;
        }
        // even row j: colours 0 and 1 from the old rows j-1 and j+1
        long long ue = rc;
        if (j >= 1 && j < q.ny) colour_pair_gs(ue, od_old + rp, ge, xin, x);
        // odd row j-1: colours 2 and 3 from the new rows j-2 and j
        if (j - 1 >= js + 1) {
          long long uo = od_old;
          if (j - 1 < q.ny) colour_pair_gs(uo, ev_new + ue, go, xin, x);
          put(j - 1, uo);
        }
        if (j < je || je == q.ny) put(j, ue);
        ev_new = ue;
        od_old = rp;
      }
    }
  }
  // block max of |new values| -> FP64 bits -> the next sweep's bound
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long w = __shfl_xor_sync(0xffffffffu, vmax, o);
    vmax = w > vmax ? w : vmax;
  }
  if (lane == 0) red[wib] = vmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long m = 0;
    for (int w = 0; w < W2_THREADS / 32; ++w) m = red[w] > m ? red[w] : m;
    atomicMax(&bnd->umax[(sweep + 1) % 4], fx::abs_bits(fx::to_double(m, R - fx::FRAC) * (1.0 + 0x1p-50)));
  }
}

// Multi-sweep damped Jacobi in the same global-scale fixed point (0 < omega <= 1):
//   u' = u + omega (3/8 h^2 f + N/8 - u),
// with omega applied as an integer product: floor(D * Wq / 2^62), Wq = omega 2^62
// rounded, exact to one unit of the last fixed-point place.  |u'| <= max|u| +
// omega 3/8 h^2 max|f|, within the bound of sweep_bounds.cuh.  If the plan rules out
// fixed point, every sweep of the call runs the FP64-capable single-sweep path on FP64
// buffers.
__device__ __forceinline__ long long omega_times(long long D, long long Wq) {
  const long long hi = __mul64hi(D, Wq);
  const unsigned long long lo = (unsigned long long)D * (unsigned long long)Wq;
  return (long long)(((unsigned long long)hi << 2) | (lo >> 62));
}

template <int XF, int YF>
__global__ void __launch_bounds__(W2_THREADS) k_jac2_sweep(Geo q, const void *__restrict__ X, void *__restrict__ Y,
                                                           const double *__restrict__ f,
                                                           const long long *__restrict__ GF, SweepBounds *bnd,
                                                           int sweep, int sweeps, double g, double omega,
                                                           long long Wq, bool write_bnd) {
  __shared__ long long red[W2_THREADS / 32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * (W2_THREADS / 32) + wib;
  const Plan plan = make_plan(bnd, g, sweeps);
  if (!plan.fix) {
    Op2Args a{};
    a.q = q;
    a.u = (const double *)X;
    a.f = f;
    a.out = (double *)Y;
    a.c1 = omega * g;
    a.c2 = -omega * 0.375 / 3.0;
    Stream2 s;
    ops2_warp<O2_JACOBI>(a, lane, gw, s, S2_ROWS);
    return;
  }
  const int R = sweep_R(bnd, sweep % 4, g);
  const int Rx = sweep > 0 ? sweep_R(bnd, (sweep + 3) % 4, g) : R;
  const int dx = XF == SF_FXP ? R - Rx : 0, df = R - plan.Rf, rb = 1023 + R;
  const int dxr = dx > 0 ? (dx < 63 ? dx : 63) : 0, dxl = dx < 0 ? (-dx < 63 ? -dx : 63) : 0;
  const int dfr = df < 63 ? df : 63;
  if (blockIdx.x == 0 && threadIdx.x == 0) bnd->umax[(sweep + 2) % 4] = 0ull;
  const int64_t nseg = (q.nx + 30) / 30;
  const int64_t seg = gw % nseg, chunk = gw / nseg;
  const int64_t js = chunk * S2_ROWS;
  long long vmax = 0;
  if (js <= q.ny) {
    const int64_t je = js + S2_ROWS < q.ny + 1 ? js + S2_ROWS : q.ny + 1;
    const int64_t x = seg * 30 + lane - 1;
    const bool xok = x >= 0 && x <= q.nx, xin = x >= 1 && x < q.nx;
    const bool out_lane = lane >= 1 && lane <= 30 && xok;
    const long long *Xl = (const long long *)X;
    auto rawx = [&](int64_t j) -> long long { return (xok && j >= 0 && j <= q.ny) ? Xl[j * q.pitch + x] : 0ll; };
    auto rawg = [&](int64_t j) -> long long { return (xin && j >= 1 && j < q.ny) ? GF[j * q.pitch + x] : 0ll; };
    auto cvx = [&](long long raw) -> long long {
      return XF == SF_F64 ? fx::to_fixed(__longlong_as_double(raw), rb) : (raw >> dxr) << dxl;
    };
    long long um = cvx(rawx(js - 1)), uc = cvx(rawx(js)), up = cvx(rawx(js + 1));
    constexpr int PQ = 3;
    long long qx[PQ], qg[PQ];  // raw X row j + 2 and GF row j for the iteration j = jb + t
#pragma unroll
    for (int t = 0; t < PQ; ++t) {
      qx[t] = rawx(js + 2 + t);
      qg[t] = rawg(js + t);
    }
    for (int64_t jb = js; jb < je; jb += PQ) {
#pragma unroll
      for (int t = 0; t < PQ; ++t) {
        const int64_t j = jb + t;
        if (j >= je) break;
        const long long rn = qx[t], gr = qg[t];
        qx[t] = j + 2 + PQ <= je ? rawx(j + 2 + PQ) : 0ll;
        qg[t] = j + PQ < je ? rawg(j + PQ) : 0ll;
        const long long V = um + up, T = V + uc;
        const long long Tm = __shfl_up_sync(0xffffffffu, T, 1);
        const long long Tp = __shfl_down_sync(0xffffffffu, T, 1);
        if (out_lane) {
          const bool inner = xin && j >= 1 && j < q.ny;
          long long un = uc;  // Dirichlet value carried
          if (inner) un = uc + omega_times((gr >> dfr) + ((Tm + Tp + V) >> 3) - uc, Wq);
          if (inner || write_bnd) {
            if (YF == SF_FXP)
              ((long long *)Y)[j * q.pitch + x] = un;
            else
              ((double *)Y)[j * q.pitch + x] = fx::to_double_cvt(un, R - fx::FRAC);
            const long long aa = un < 0 ? -un : un;
            vmax = aa > vmax ? aa : vmax;
          }
        }
        um = uc;
        uc = up;
        up = cvx(rn);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long w = __shfl_xor_sync(0xffffffffu, vmax, o);
    vmax = w > vmax ? w : vmax;
  }
  if (lane == 0) red[wib] = vmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long m = 0;
    for (int w = 0; w < W2_THREADS / 32; ++w) m = red[w] > m ? red[w] : m;
    atomicMax(&bnd->umax[(sweep + 1) % 4], fx::abs_bits(fx::to_double(m, R - fx::FRAC) * (1.0 + 0x1p-50)));
  }
}

}  // namespace

size_t ops2_reduce_bytes(const Geo &q) { return 16 + (size_t)ops2_blocks(q) * 2 * sizeof(double); }

static cudaError_t launch_ops2(int op, const Op2Args &a, cudaStream_t s) {
  const unsigned nb = ops2_blocks(a.q);
  switch (op) {
    case O2_APPLY: k_ops2<O2_APPLY><<<nb, W2_THREADS, 0, s>>>(a); break;
    case O2_JACOBI: k_ops2<O2_JACOBI><<<nb, W2_THREADS, 0, s>>>(a); break;
    case O2_RESIDUAL: k_ops2<O2_RESIDUAL><<<nb, W2_THREADS, 0, s>>>(a); break;
    default: k_ops2<O2_ELEMENTWISE><<<nb, W2_THREADS, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_apply_fx2(const Geo &q, const double *u, double *y, bool elementwise, cudaStream_t s) {
  Op2Args a{};
  a.q = q;
  a.u = u;
  a.out = y;
  a.c1 = elementwise ? 1.0 / (6.0 * q.h * q.h) : 1.0 / (3.0 * q.h * q.h);
  return launch_ops2(elementwise ? O2_ELEMENTWISE : O2_APPLY, a, s);
}

cudaError_t launch_jacobi_fx2(const Geo &q, const double *u, const double *f, double *unew, double omega,
                              cudaStream_t s) {
  Op2Args a{};
  a.q = q;
  a.u = u;
  a.f = f;
  a.out = unew;
  a.c1 = omega * 0.375 * q.h * q.h;
  a.c2 = -omega * 0.375 / 3.0;
  return launch_ops2(O2_JACOBI, a, s);
}

cudaError_t launch_residual_fx2(const Geo &q, const double *u, const double *f, double *r, double *norms2,
                                void *scratch, cudaStream_t s) {
  Op2Args a{};
  a.q = q;
  a.u = u;
  a.f = f;
  a.out = r;
  a.c1 = -1.0 / (3.0 * q.h * q.h);
  a.counter = (unsigned *)scratch;
  a.partials = (double *)((char *)scratch + 16);
  a.norms2 = norms2;
  return launch_ops2(O2_RESIDUAL, a, s);
}

// work: 3 arrays of u's span (8 bytes per element): two int64 ping-pong buffers and
// GF; bounds: gs_fx_bounds_bytes() bytes.  The result always ends in u, whose boundary
// values are never written.
cudaError_t launch_gs_sweeps_fx2(const Geo &q, double *u, const double *f, int sweeps, double *work, void *bounds,
                                 cudaStream_t s) {
  const double g = 0.375 * q.h * q.h;
  const int64_t nseg = (q.nx + 24) / 24;
  const int64_t nchunk = (q.ny + S2_ROWS) / S2_ROWS;
  const unsigned nb = (unsigned)((nseg * nchunk + W2_THREADS / 32 - 1) / (W2_THREADS / 32));
  const int64_t span = span_elems(q);
  cudaError_t e;
  if (sweeps == 1) {
    k_gs2_fused<<<nb, W2_THREADS, 0, s>>>(q, u, work, f, g);
    e = cudaGetLastError();
    return e ? e : cudaMemcpyAsync(u, work, (size_t)span * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  void *A = work, *B = work + span;
  long long *GF = (long long *)(work + 2 * span);
  SweepBounds *bnd = (SweepBounds *)bounds;
  e = launch_gs_prepass(q, 2, u, f, GF, bounds, sweeps, s);
  const void *X = u;
  for (int it = 0; it < sweeps && !e; ++it) {
    const bool first = it == 0, last = it == sweeps - 1;
    void *Y = last ? (void *)u : (it % 2 == 0 ? A : B);
    if (first)
      k_gs2_sweep<SF_F64, SF_FXP><<<nb, W2_THREADS, 0, s>>>(q, X, Y, f, GF, bnd, it, sweeps, g, true);
    else if (!last)
      k_gs2_sweep<SF_FXP, SF_FXP><<<nb, W2_THREADS, 0, s>>>(q, X, Y, f, GF, bnd, it, sweeps, g, true);
    else  // the caller's u: its Dirichlet values were never overwritten, leave them
      k_gs2_sweep<SF_FXP, SF_F64><<<nb, W2_THREADS, 0, s>>>(q, X, Y, f, GF, bnd, it, sweeps, g, false);
    e = cudaGetLastError();
    X = Y;
  }
  return e;
}

}  // namespace stencil

namespace stencil {

// Multi-sweep damped Jacobi, 2D, 0 < omega <= 1.  A: u-sized buffer (the caller's
// work array); scratch: 2 u-sized buffers (second ping-pong buffer and GF); bounds:
// gs_fx_bounds_bytes().  The result ends in u; u's boundary is never written.
cudaError_t launch_jacobi_sweeps_fx2(const Geo &q, double *u, const double *f, int sweeps, double omega, double *A,
                                     double *scratch, void *bounds, cudaStream_t s) {
  const double g = 0.375 * q.h * q.h;
  const int64_t nseg = (q.nx + 30) / 30;
  const int64_t nchunk = (q.ny + S2_ROWS) / S2_ROWS;
  const unsigned nb = (unsigned)((nseg * nchunk + W2_THREADS / 32 - 1) / (W2_THREADS / 32));
  const int64_t span = span_elems(q);
  void *B = scratch;
  long long *GF = (long long *)(scratch + span);
  SweepBounds *bnd = (SweepBounds *)bounds;
  const long long Wq = (long long)llrint(omega * 0x1p62);
  if (sweeps == 1) {  // u -> A (boundary copied), then back
    cudaError_t e = launch_jacobi_fx2(q, u, f, A, omega, s);
    return e ? e : cudaMemcpyAsync(u, A, (size_t)span * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  cudaError_t e = launch_gs_prepass(q, 2, u, f, GF, bounds, sweeps, s);
  const void *X = u;
  for (int it = 0; it < sweeps && !e; ++it) {
    const bool first = it == 0, last = it == sweeps - 1;
    void *Y = last ? (void *)u : (it % 2 == 0 ? (void *)A : B);
    if (first)
      k_jac2_sweep<SF_F64, SF_FXP><<<nb, W2_THREADS, 0, s>>>(q, X, Y, f, GF, bnd, it, sweeps, g, omega, Wq, true);
    else if (!last)
      k_jac2_sweep<SF_FXP, SF_FXP><<<nb, W2_THREADS, 0, s>>>(q, X, Y, f, GF, bnd, it, sweeps, g, omega, Wq, true);
    else
      k_jac2_sweep<SF_FXP, SF_F64><<<nb, W2_THREADS, 0, s>>>(q, X, Y, f, GF, bnd, it, sweeps, g, omega, Wq, false);
    e = cudaGetLastError();
    X = Y;
  }
  return e;
}

}  // namespace stencil
