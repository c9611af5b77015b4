// 2D Q1 (bilinear, 9-point stencil of Fig. 1) operations on the integer pipes:
// assembled apply, element-wise apply with colour passes, damped Jacobi sweeps,
// residual with norms, and coloured Gauss-Seidel sweeps (the multi-sweep smoothers run
// two sweeps per pass over memory).
//
//   3 S u = 8 u - N,  N = sum of the 8 neighbours;   6 K_e (element matrix, h-free) has
//   entries 4 (same vertex), -1 (differ in one coordinate), -2 (opposite corner).
// Values are int64 fixed point (fixed.cuh); N is formed from column sums
//   V = u(j-1) + u(j+1),  T = V + u(j),  N(x) = T(x-1) + T(x+1) + V(x).
//
// Each warp owns a window of 64 consecutive columns, two per lane (an even and an odd
// x), and streams down a chunk of rows, keeping the rows it needs in registers and
// reaching x-neighbours by shuffles; no shared memory and no block barriers (the
// single-sweep FP64-adaptive Gauss-Seidel kernel keeps one column per lane).  Rows move
// as 16-byte pairs where the arrays are 16-byte aligned with an even pitch.  For the
// single-pass operations the fixed-point
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
// CTAs per SM the two-sweep kernels are compiled for: with 5 the GS kernel fits in 96
// registers instead of 106 (4 CTAs per SM), one more CTA of warps to hide the latency
// of the row fronts (measured at 16385^2: GS 40.1 -> 37.5 ms and Jacobi 43.6 ->
// 42.7 ms per 50 sweeps; 6, at 80 registers, spills and is slower)
constexpr int S2X2_MIN_CTAS = 5;
constexpr int R_MIN = -900, R_MAX = 1000;

enum { O2_APPLY = 0, O2_JACOBI = 1, O2_RESIDUAL = 2, O2_ELEMENTWISE = 3 };

// Per operation: convert the fixed-point result with the FP64 pipe (true) or with
// integer instructions (false), whichever measured faster (the element-wise apply
// always uses the FP64 pipe).
constexpr bool OP2_CVT[4] = {true, true, false, true};

// With OP2_CVT: the odd-x column of each lane pair converts with integer instructions
// instead (true), which moves a quarter of the FP64-pipe work of the conversions onto
// the integer pipes; both give the same bits.
constexpr bool OP2_SPLIT[4] = {true, false, false, false};

// Per assembled operation: compute on the halo lanes too instead of branching around
// them (true), whichever measured faster.
constexpr bool OP2_NOBRANCH[4] = {false, false, true, false};

struct Op2Args {
  Geo q;
  const double *u, *f;
  double *out;
  double c1, c2;
  double *partials;
  unsigned *counter;
  double *norms2;
  int rows;  // rows per warp (W2_ROWS unless a tuned shape says otherwise)
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

// ------------------------------------------------------------------ lane pairs
// Each lane owns two adjacent columns, xa (even x) and xb = xa + 1, of its warp's
// 64-column window; rows move as 16-byte pairs when the arrays allow it (V16: 16-byte
// aligned bases, even pitch).  A neighbour across the pair boundary comes from the
// adjacent lane by one 64-bit shuffle.
struct Pair {
  long long a, b;  // columns xa (even x) and xb (odd x)
};

// Columns of one lane and their validity.
struct Cols {
  int64_t xa;
  bool oka, okb;  // inside the row (0 <= x <= nx)
  bool ina, inb;  // interior column (1 <= x < nx)
};

__device__ __forceinline__ Cols make_cols(const Geo &q, int64_t xa) {
  Cols c;
  c.xa = xa;
  c.oka = xa >= 0 && xa <= q.nx;
  c.okb = xa + 1 >= 0 && xa + 1 <= q.nx;
  c.ina = xa >= 1 && xa < q.nx;
  c.inb = xa + 1 >= 1 && xa + 1 < q.nx;
  return c;
}

// Raw 64-bit pair of row pointer `row` (zeros outside the row).
template <bool V16>
__device__ __forceinline__ Pair ld_pair(const long long *__restrict__ row, const Cols &c) {
  Pair p{0ll, 0ll};
  if (V16 && c.oka && c.okb) {
    const longlong2 v = *(const longlong2 *)(row + c.xa);
    p.a = v.x;
    p.b = v.y;
  } else {
    if (c.oka) p.a = row[c.xa];
    if (c.okb) p.b = row[c.xa + 1];
  }
  return p;
}

template <bool V16>
__device__ __forceinline__ void st_pair(long long *__restrict__ row, const Cols &c, bool wa, bool wb, long long a,
                                        long long b) {
  if (V16 && wa && wb) {
    *(longlong2 *)(row + c.xa) = make_longlong2(a, b);
  } else {
    if (wa) row[c.xa] = a;
    if (wb) row[c.xa + 1] = b;
  }
}

__device__ __forceinline__ unsigned pair_exp(const Pair &r) {
  return max(biased_exp(__longlong_as_double(r.a)), biased_exp(__longlong_as_double(r.b)));
}

template <bool FIX>
__device__ __forceinline__ Pair pair_in(const Pair &raw, const WarpScale &w) {
  if (!FIX) return raw;
  return Pair{fx::to_fixed(__longlong_as_double(raw.a), 1023 + w.R), fx::to_fixed(__longlong_as_double(raw.b), 1023 + w.R)};
}

__device__ __forceinline__ Pair pair_shr(const Pair &p, int d) { return Pair{shr(p.a, d), shr(p.b, d)}; }

__device__ __forceinline__ Pair pair_f64(const Pair &p, int R) { return Pair{to_f64_bits(p.a, R), to_f64_bits(p.b, R)}; }

// 8u - N (3 S u) at both columns from the rows above (m), at (c) and below (p):
//   V = m + p,  T = V + c,  N(x) = (T(x-1) + T(x+1)) + V(x).
template <bool FIX>
__device__ __forceinline__ Pair eight_u_minus_n(const Pair &m, const Pair &c, const Pair &p) {
  const Pair V{add<FIX>(m.a, p.a), add<FIX>(m.b, p.b)};
  const Pair T{add<FIX>(V.a, c.a), add<FIX>(V.b, c.b)};
  const long long Tbl = __shfl_up_sync(0xffffffffu, T.b, 1);   // T(xa - 1)
  const long long Tar = __shfl_down_sync(0xffffffffu, T.a, 1); // T(xb + 1)
  const long long Na = add<FIX>(add<FIX>(Tbl, T.b), V.a), Nb = add<FIX>(add<FIX>(T.a, Tar), V.b);
  if (FIX) return Pair{8 * c.a - Na, 8 * c.b - Nb};
  return Pair{__double_as_longlong(fma(8.0, __longlong_as_double(c.a), -__longlong_as_double(Na))),
              __double_as_longlong(fma(8.0, __longlong_as_double(c.b), -__longlong_as_double(Nb)))};
}

constexpr int PF = 2;      // rows in flight per warp (assembled operations)
constexpr int PF_EW = 1;   // rows in flight per warp (element-wise apply; measured faster)
// Element-wise apply: every lane evaluates both of its cells in a cell row inside the
// grid, also a cell beyond the last column (its shares land only on boundary vertices,
// whose output is 0, or on columns that are not written): no divergent branch per cell.
constexpr bool EW2_ALLCELLS = true;
constexpr int OPS2_OUT = 60;  // output columns per warp: lanes 1..30 (one halo column per side)

// Per-warp streaming state of k_ops2.
struct Stream2 {
  Cols c;
  bool out_lane;
  int lane;
  Pair um, uc, up;  // converted rows j-1, j, j+1 (element-wise: ua = uc, accumulators um/up)
  Pair rc, rp;      // raw rows j, j+1 (FP64 bits)
  double rr, ff;
};

// Element matrix 6 K_e of one cell times its vertex values v0 = (x, y), v1 = (x+1, y),
// v2 = (x, y+1), v3 = (x+1, y+1): 4 v_w - (the two face-adjacent values) - 2 v_opposite
// (the FP64 path; the fixed-point path forms the same sums as in ew2_rows).
template <bool FIX>
__device__ __forceinline__ void cell_contrib(long long v0, long long v1, long long v2, long long v3, long long &c0,
                                             long long &c1, long long &c2, long long &c3) {
  if (FIX) {
    const long long s1 = v1 + v2, s2 = v0 + v3;
    c0 = 4 * v0 - s1 - 2 * v3;
    c1 = 4 * v1 - s2 - 2 * v2;
    c2 = 4 * v2 - s2 - 2 * v1;
    c3 = 4 * v3 - s1 - 2 * v0;
  } else {
    const double A0 = __longlong_as_double(v0), A1 = __longlong_as_double(v1), A2 = __longlong_as_double(v2),
                 A3 = __longlong_as_double(v3);
    c0 = __double_as_longlong(4.0 * A0 - (A1 + A2) - 2.0 * A3);
    c1 = __double_as_longlong(4.0 * A1 - (A0 + A3) - 2.0 * A2);
    c2 = __double_as_longlong(4.0 * A2 - (A0 + A3) - 2.0 * A1);
    c3 = __double_as_longlong(4.0 * A3 - (A1 + A2) - 2.0 * A0);
  }
}

// Element-wise apply: cell rows cj in [cj0, je); returns the first row not done (a
// switch to FP64 was requested) or je.  The lane's cells are A (lower-left vertex xa:
// all four vertices in this lane) and B (lower-left vertex xb: its right vertices are
// the next lane's xa).  Each vertex column is owned by one lane, which adds the shares
// of the cells on both of its sides (B of the lane to the left arrives by shuffle), so
// the scatter has no write conflicts.  In fixed point the sums are exact, so the order
// of the two x colours is immaterial; the FP64 path adds the even-x colour's share
// first.
template <bool FIX, bool V16>
__device__ __forceinline__ int64_t ew2_rows(const Op2Args &a, WarpScale &w, Stream2 &s, int64_t cj0, int64_t js,
                                            int64_t je) {
  const Geo &q = a.q;
  const Cols &c = s.c;
  const long long *ub_ = (const long long *)a.u;
  Pair &ua = s.uc, &alo = s.um, &ahi = s.up;
  // output scale c1 2^(R-52), re-formed only when R changes (an FP64 multiply per
  // output would otherwise load the FP64 pipe, this kernel's bottleneck)
  double sc = FIX ? a.c1 * fx::pow2d(w.R - fx::FRAC) : a.c1;
  auto raw = [&](int64_t j) -> Pair {
    return (j >= 0 && j <= q.ny) ? ld_pair<V16>(ub_ + j * q.pitch, c) : Pair{0ll, 0ll};
  };
  Pair qb[PF_EW];  // qb[t]: raw vertex row cj + 1 for the iteration cj = cb + t
#pragma unroll
  for (int t = 0; t < PF_EW; ++t) qb[t] = raw(cj0 + 1 + t);
  for (int64_t cb = cj0; cb < je; cb += PF_EW) {
#pragma unroll
    for (int t = 0; t < PF_EW; ++t) {
      const int64_t cj = cb + t;
      if (cj >= je) return je;
      const Pair rb = qb[t];
      const unsigned em = __reduce_max_sync(0xffffffffu, pair_exp(rb));
      if (FIX) {
        const int d = admit_row(w, em, 1);
        if (d < 0) {  // leave this row to the FP64 loop
          if (cj >= 1) alo = Pair{alo.a + 12 * ua.a, alo.b + 12 * ua.b};  // the 6 u_v of cell row cj - 1
          ua = pair_f64(ua, w.R);
          alo = pair_f64(alo, w.R);
          ahi = pair_f64(ahi, w.R);
          w.fix = false;
          return cj;
        }
        if (d > 0) {
          ua = pair_shr(ua, d);
          alo = pair_shr(alo, d);
          ahi = pair_shr(ahi, d);
          sc = a.c1 * fx::pow2d(w.R - fx::FRAC);
        }
      }
      qb[t] = cj + 1 + PF_EW <= je ? raw(cj + 1 + PF_EW) : Pair{0ll, 0ll};
      const Pair ub = pair_in<FIX>(rb, w);
      const long long uar = __shfl_down_sync(0xffffffffu, ua.a, 1);  // (xb + 1, cj)
      const long long ubr = __shfl_down_sync(0xffffffffu, ub.a, 1);  // (xb + 1, cj + 1)
      const bool crow = cj >= 0 && cj < q.ny;
      const bool cellA = crow && c.xa >= 0 && c.xa < q.nx;
      const bool cellB = crow && s.lane <= 30 && c.xa + 1 >= 0 && c.xa + 1 < q.nx;
      if (FIX) {
        // 6 K_e u_e at a vertex of the cell = 6 u_v - d, d = s + 2 s' with s the sum of
        // the vertex's two edge neighbours in the cell and s' the sum of the vertex and
        // its opposite: one d for each diagonal pair of the cell.  The 6 u_v parts of the
        // vertex's four cells are added once, as 24 u_v, when the row is complete.
        long long dA03 = 0, dA12 = 0, dB03 = 0, dB12 = 0;
        if (EW2_ALLCELLS ? crow : cellA) {
          const long long s12 = ua.b + ub.a, s03 = ua.a + ub.b;
          dA03 = s12 + 2 * s03;
          dA12 = s03 + 2 * s12;
        }
        if (EW2_ALLCELLS ? crow : cellB) {
          const long long s12 = uar + ub.b, s03 = ua.b + ubr;
          dB03 = s12 + 2 * s03;
          dB12 = s03 + 2 * s12;
        }
        long long dB12l = __shfl_up_sync(0xffffffffu, dB12, 1), dB03l = __shfl_up_sync(0xffffffffu, dB03, 1);
        if (s.lane == 0) dB12l = dB03l = 0;
        alo.a -= dA03 + dB12l;
        ahi.a -= dA12 + dB03l;
        alo.b -= dA12 + dB03;
        ahi.b -= dA03 + dB12;
      } else {
        long long a0 = 0, a1 = 0, a2 = 0, a3 = 0, b0 = 0, b1 = 0, b2 = 0, b3 = 0;
        if (EW2_ALLCELLS ? crow : cellA) cell_contrib<FIX>(ua.a, ua.b, ub.a, ub.b, a0, a1, a2, a3);
        if (EW2_ALLCELLS ? crow : cellB) cell_contrib<FIX>(ua.b, uar, ub.b, ubr, b0, b1, b2, b3);
        long long b1l = __shfl_up_sync(0xffffffffu, b1, 1), b3l = __shfl_up_sync(0xffffffffu, b3, 1);
        if (s.lane == 0) b1l = b3l = 0;
        // vertex xa: cell A (even x) then the left lane's cell B; vertex xb: A then B
        alo.a = add<FIX>(add<FIX>(alo.a, a0), b1l);
        ahi.a = add<FIX>(add<FIX>(ahi.a, a2), b3l);
        alo.b = add<FIX>(add<FIX>(alo.b, a1), b0);
        ahi.b = add<FIX>(add<FIX>(ahi.b, a3), b2);
      }
      if (cj >= js) {
        const bool jin = cj >= 1 && cj < q.ny;
        // FIX: the converted sum times c1 2^(R-52) (exact power-of-two scaling of c1)
        constexpr bool SPLIT = OP2_SPLIT[O2_ELEMENTWISE];
        const long long sa = FIX ? alo.a + 24 * ua.a : alo.a, sbv = FIX ? alo.b + 24 * ua.b : alo.b;
        const double va = FIX ? __ll2double_rn(sa) : __longlong_as_double(sa);
        const double vb = !FIX ? __longlong_as_double(sbv)
                          : SPLIT ? fx::to_double(sbv, w.R - fx::FRAC) : __ll2double_rn(sbv);
        const double sb = FIX && SPLIT ? a.c1 : sc;
        st_pair<V16>((long long *)a.out + cj * q.pitch, c, s.out_lane && c.oka, s.out_lane && c.okb,
                     __double_as_longlong(jin && c.ina ? va * sc : 0.0),
                     __double_as_longlong(jin && c.inb ? vb * sb : 0.0));
      }
      alo = ahi;
      ahi = Pair{0ll, 0ll};
      ua = ub;
    }
  }
  return je;
}

// Assembled apply / Jacobi / residual: output rows j in [j0, je).
template <bool FIX, int OP, bool V16>
__device__ __forceinline__ int64_t op2_rows(const Op2Args &a, WarpScale &w, Stream2 &s, int64_t j0, int64_t js,
                                            int64_t je) {
  const Geo &q = a.q;
  const Cols &c = s.c;
  const long long *ub_ = (const long long *)a.u;
  const long long *fb_ = (const long long *)a.f;
  long long *ob_ = (long long *)a.out;
  // CVT: T is converted by the FP64 pipe and multiplied by the factor of its term times
  // 2^(R-52) (re-formed only when R changes); otherwise by fx::to_double on the integer
  // pipe.  Both give the same bits.
  constexpr bool CVT = OP2_CVT[OP], CVTB = CVT && !OP2_SPLIT[OP];
  const double cf = OP == O2_JACOBI ? a.c2 : a.c1;  // factor of the converted term
  double sc = FIX && CVT ? cf * fx::pow2d(w.R - fx::FRAC) : cf;
  const double scb_int = cf;  // the odd column's factor when it converts on the integer pipe
  auto scb = [&]() -> double { return FIX && !CVTB ? scb_int : sc; };
  auto raw = [&](int64_t j) -> Pair {
    return (j >= 0 && j <= q.ny) ? ld_pair<V16>(ub_ + j * q.pitch, c) : Pair{0ll, 0ll};
  };
  Pair qb[PF];  // qb[t]: raw row j + 2 for the iteration j = jb + t
#pragma unroll
  for (int t = 0; t < PF; ++t) qb[t] = raw(j0 + 2 + t);
  for (int64_t jb = j0; jb < je; jb += PF) {
#pragma unroll
    for (int t = 0; t < PF; ++t) {
      const int64_t j = jb + t;
      if (j >= je) return je;
      const Pair rn = qb[t];  // row j + 2
      const unsigned em = __reduce_max_sync(0xffffffffu, pair_exp(rn));
      const bool jin = j >= 1 && j < q.ny;
      Pair fv{0ll, 0ll};  // FP64 bits
      if (OP != O2_APPLY && s.out_lane && jin) fv = ld_pair<V16>(fb_ + j * q.pitch, c);
      const Pair T = eight_u_minus_n<FIX>(s.um, s.uc, s.up);
      constexpr bool NB = OP2_NOBRANCH[OP];
      if (NB || s.out_lane) {
        // OP2_NOBRANCH: every lane computes (no branch around the halo lanes); only
        // output lanes store
        const bool ia = jin && c.ina && s.out_lane, ib = jin && c.inb && s.out_lane;
        // Td * sc == T's value times the term's factor
        auto conv = [&](long long v, bool cvt) -> double {
          return !FIX ? __longlong_as_double(v) : cvt ? __ll2double_rn(v) : fx::to_double(v, w.R - fx::FRAC);
        };
        const double Ta = conv(T.a, CVT), Tb = conv(T.b, CVTB);
        const double sb = scb();
        const double fa = __longlong_as_double(fv.a), fb = __longlong_as_double(fv.b);
        const double rca = __longlong_as_double(s.rc.a), rcb = __longlong_as_double(s.rc.b);
        double oa, ob;
        if (OP == O2_APPLY) {
          oa = ia ? Ta * sc : 0.0;
          ob = ib ? Tb * sb : 0.0;
        } else if (OP == O2_JACOBI) {
          oa = ia ? fma(sc, Ta, fma(a.c1, fa, rca)) : rca;
          ob = ib ? fma(sb, Tb, fma(a.c1, fb, rcb)) : rcb;
        } else {
          oa = ia ? fma(sc, Ta, fa) : 0.0;
          ob = ib ? fma(sb, Tb, fb) : 0.0;
          if (ia) {
            s.rr = fma(oa, oa, s.rr);
            s.ff = fma(fa, fa, s.ff);
          }
          if (ib) {
            s.rr = fma(ob, ob, s.rr);
            s.ff = fma(fb, fb, s.ff);
          }
        }
        if (OP != O2_RESIDUAL || ob_)
          st_pair<V16>(ob_ + j * q.pitch, c, s.out_lane && c.oka, s.out_lane && c.okb, __double_as_longlong(oa),
                       __double_as_longlong(ob));
      }
      // admit row j + 2 (after row j is done)
      if (FIX) {
        const int d = admit_row(w, em, 1);
        if (d < 0) {
          s.uc = pair_f64(s.uc, w.R);
          s.up = pair_f64(s.up, w.R);
          w.fix = false;
          // row j is finished; rows j+1, j+2 continue in FP64 (rn still in the queue)
          s.um = s.uc;
          s.uc = s.up;
          s.up = rn;
          s.rc = s.rp;
          s.rp = rn;
          return j + 1;
        }
        if (d > 0) {
          s.uc = pair_shr(s.uc, d);
          s.up = pair_shr(s.up, d);
          if (CVT) sc = cf * fx::pow2d(w.R - fx::FRAC);
        }
      }
      qb[t] = j + 2 + PF <= je ? raw(j + 2 + PF) : Pair{0ll, 0ll};
      s.um = s.uc;
      s.uc = s.up;
      s.up = pair_in<FIX>(rn, w);
      s.rc = s.rp;
      s.rp = rn;
    }
  }
  return je;
}

// Work units of the single-pass 2D operations: 60-column segments x chunks of `rows`.
__host__ __device__ __forceinline__ int64_t ops2_units(const Geo &q, int rows) {
  return (int64_t)((q.nx + OPS2_OUT) / OPS2_OUT) * ((q.ny + rows) / rows);
}

// One warp's share of k_ops2: a segment of 60 output columns and a chunk of rows.
template <int OP, bool V16>
__device__ __forceinline__ void ops2_warp(const Op2Args &a, int lane, int64_t gw, Stream2 &s, int rows) {
  const Geo &q = a.q;
  const int64_t nseg = (q.nx + OPS2_OUT) / OPS2_OUT;
  const int64_t seg = gw % nseg, chunk = gw / nseg;
  const int64_t js = chunk * rows;
  const int64_t je = js + rows < q.ny + 1 ? js + rows : q.ny + 1;
  s.lane = lane;
  s.c = make_cols(q, seg * OPS2_OUT - 2 + 2 * lane);  // lanes 1..30 produce outputs
  s.out_lane = lane >= 1 && lane <= 30;
  s.rr = 0.0;
  s.ff = 0.0;
  WarpScale w;
  if (js <= q.ny) {
    const long long *ub_ = (const long long *)a.u;
    auto load = [&](int64_t j) -> Pair {
      return (j >= 0 && j <= q.ny) ? ld_pair<V16>(ub_ + j * q.pitch, s.c) : Pair{0ll, 0ll};
    };
    if (OP == O2_ELEMENTWISE) {
      const Pair ra = load(js - 1);
      if (admit_row(w, __reduce_max_sync(0xffffffffu, pair_exp(ra)), 1) < 0) w.fix = false;
      s.uc = w.fix ? pair_in<true>(ra, w) : ra;
      s.um = Pair{0ll, 0ll};
      s.up = Pair{0ll, 0ll};
      int64_t cj = js - 1;
      if (w.fix) cj = ew2_rows<true, V16>(a, w, s, cj, js, je);
      if (cj < je) ew2_rows<false, V16>(a, w, s, cj, js, je);
    } else {
      s.rc = load(js);
      s.rp = load(js + 1);
      const Pair rm = load(js - 1);
      unsigned em = __reduce_max_sync(0xffffffffu, pair_exp(rm));
      em = max(em, __reduce_max_sync(0xffffffffu, pair_exp(s.rc)));
      em = max(em, __reduce_max_sync(0xffffffffu, pair_exp(s.rp)));
      if (admit_row(w, em, 1) < 0) w.fix = false;
      s.um = w.fix ? pair_in<true>(rm, w) : rm;
      s.uc = w.fix ? pair_in<true>(s.rc, w) : s.rc;
      s.up = w.fix ? pair_in<true>(s.rp, w) : s.rp;
      int64_t j = js;
      if (w.fix) j = op2_rows<true, OP, V16>(a, w, s, j, js, je);
      if (j < je) op2_rows<false, OP, V16>(a, w, s, j, js, je);
    }
  }
}

template <int OP, bool V16>
__global__ void __launch_bounds__(W2_THREADS) k_ops2(Op2Args a) {
  __shared__ double sh[2 * W2_THREADS / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  Stream2 s;
  ops2_warp<OP, V16>(a, lane, (int64_t)blockIdx.x * (W2_THREADS / 32) + wib, s, a.rows);
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

unsigned ops2_blocks(const Geo &q, int rows) {
  return (unsigned)((ops2_units(q, rows) + W2_THREADS / 32 - 1) / (W2_THREADS / 32));
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
// last store into u.
//
// Each lane owns two adjacent columns, xa (even x) and xb = xa + 1 (odd x), so a colour
// step that updates one x parity touches exactly one of the lane's columns and takes
// one neighbour from an adjacent lane (one 64-bit shuffle); rows move as 16-byte
// pairs when the arrays allow it (V16: 16-byte aligned base, even pitch).
enum { SF_F64 = 0, SF_FXP = 1 };  // storage format: FP64, or int64 fixed point

// High word of |v| (ones' complement: |v| or |v| - 1), an upper bound of |v| / 2^32 - 1
// in 3 integer instructions; the sweeps track max |u| through it.
__device__ __forceinline__ unsigned mag_hi(long long v) {
  const int hi = (int)(v >> 32);
  return (unsigned)(hi ^ (hi >> 31));
}

// Store one row pair of the new iterate (fixed point, or FP64 for the call's last
// sweep) and fold its magnitude into hmax.
template <int YF, bool V16>
__device__ __forceinline__ void put_pair(const Geo &q, void *Y, int64_t j, const Cols &c, bool out_lane,
                                         bool write_bnd, int R, const Pair &v, unsigned &hmax) {
  const bool jin = j >= 1 && j < q.ny;
  const bool wa = out_lane && c.oka && ((c.ina && jin) || write_bnd);
  const bool wb = out_lane && c.okb && ((c.inb && jin) || write_bnd);
  const int64_t ro = j * q.pitch;
  if (YF == SF_FXP) {
    st_pair<V16>((long long *)Y + ro, c, wa, wb, v.a, v.b);
  } else {
    const double da = fx::to_double_cvt(v.a, R - fx::FRAC), db = fx::to_double_cvt(v.b, R - fx::FRAC);
    st_pair<V16>((long long *)Y + ro, c, wa, wb, __double_as_longlong(da), __double_as_longlong(db));
  }
  const unsigned ha = wa ? mag_hi(v.a) : 0u, hb = wb ? mag_hi(v.b) : 0u;
  hmax = max(hmax, max(ha, hb));
}

// Block max of the magnitude words -> FP64 bits -> the bound slot of the next sweep.
__device__ __forceinline__ void publish_bound(SweepBounds *bnd, int slot, int R, unsigned hmax, unsigned *red) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  hmax = __reduce_max_sync(0xffffffffu, hmax);
  if (lane == 0) red[wib] = hmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned m = 0;
    for (int w = 0; w < W2_THREADS / 32; ++w) m = red[w] > m ? red[w] : m;
    // every |v| written is < (m + 1) 2^32
    const long long ub = (long long)(((unsigned long long)m + 1ull) << 32);
    atomicMax(&bnd->umax[slot], fx::abs_bits(fx::to_double(ub, R - fx::FRAC) * (1.0 + 0x1p-50)));
  }
}

// Converts raw input values of format XF to this sweep's scale.
template <int XF>
struct InScale {
  int rb, dxr, dxl;
  __device__ __forceinline__ long long operator()(long long raw) const {
    return XF == SF_F64 ? fx::to_fixed(__longlong_as_double(raw), rb) : (raw >> dxr) << dxl;
  }
  __device__ __forceinline__ Pair operator()(const Pair &p) const { return Pair{(*this)(p.a), (*this)(p.b)}; }
};

// One colour pair of Gauss-Seidel on a row held as lane pairs: first the even-x
// column (its x-neighbours: the odd column of the lane to the left and this lane's
// odd column), then the odd-x column (this lane's new even column and the even column
// of the lane to the right).  V: sum of the rows above and below; gv: 3/8 h^2 f.
//   u_new = 3/8 h^2 f + N / 8,  N = T(x-1) + T(x+1) + V(x),  T = V + u.
__device__ __forceinline__ void gs_pair(Pair &u, const Pair &V, const Pair &gv, const Cols &c) {
  const long long Tb = V.b + u.b;
  const long long Tbl = __shfl_up_sync(0xffffffffu, Tb, 1);
  if (c.ina) u.a = gv.a + ((Tbl + Tb + V.a) >> 3);
  const long long Ta = V.a + u.a;
  const long long Tar = __shfl_down_sync(0xffffffffu, Ta, 1);
  if (c.inb) u.b = gv.b + ((Ta + Tar + V.b) >> 3);
}

// Gauss-Seidel sweep, single pass over memory (row wavefront inside a warp): for even
// row j colours 0 (x even) and 1 (x odd) from the old rows j-1, j+1; then odd row j-1,
// colours 2 and 3, from the new rows j-2 and j.  Every value read is the one the
// sequential colour order would read.  A warp covers 64 columns; each colour step
// consumes one column of halo per side, so the 56 columns of lanes 2..29 are produced.
// A chunk of rows [js, je] (js even) also recomputes its last even row je (which the
// next chunk owns) so that its last odd row can be finished; chunks are independent.
constexpr int GS2_OUT = 56;

template <int XF, int YF, bool V16>
__global__ void __launch_bounds__(W2_THREADS) k_gs2_sweep(Geo q, const void *__restrict__ X, void *__restrict__ Y,
                                                          const double *__restrict__ f,
                                                          const long long *__restrict__ GF, SweepBounds *bnd,
                                                          int sweep, int sweeps, double g, bool write_bnd, int rows) {
  __shared__ unsigned red[W2_THREADS / 32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * (W2_THREADS / 32) + wib;
  const Plan plan = make_plan(bnd, g, sweeps);
  if (!plan.fix) {
    // bound unusable for fixed point: every sweep of the call keeps FP64 buffers and
    // runs the per-warp adaptive kernel's work units (24-column segments), grid-stride
    const int64_t nseg24 = (q.nx + 24) / 24, units = nseg24 * ((q.ny + rows) / rows);
    for (int64_t w = gw; w < units; w += (int64_t)gridDim.x * (W2_THREADS / 32))
      gs2_fused_warp(q, (const double *)X, (double *)Y, f, g, w % nseg24, (w / nseg24) * rows, lane, rows);
    return;
  }
  const int R = sweep_R(bnd, sweep % 4, g);
  const int Rx = sweep > 0 ? sweep_R(bnd, (sweep + 3) % 4, g) : R;
  const int dx = XF == SF_FXP ? R - Rx : 0, df = R - plan.Rf;
  // shift amounts clamped once: inputs by dx (right, or left when the scale shrank),
  // GF by df >= 0 (a shift by 63 leaves 0 or -1: below one unit of the last place)
  InScale<XF> cvx{1023 + R, dx > 0 ? (dx < 63 ? dx : 63) : 0, dx < 0 ? (-dx < 63 ? -dx : 63) : 0};
  const int dfr = df < 63 ? df : 63;
  if (blockIdx.x == 0 && threadIdx.x == 0) bnd->umax[(sweep + 2) % 4] = 0ull;
  unsigned hmax = 0;
  const int64_t nseg = (q.nx + GS2_OUT) / GS2_OUT;
  const int64_t seg = gw % nseg, chunk = gw / nseg;
  const int64_t js = chunk * rows;  // even
  if (js <= q.ny) {
    int64_t je = js + rows;
    if (je > q.ny) je = (q.ny & 1) ? q.ny + 1 : q.ny;
    const Cols c = make_cols(q, seg * GS2_OUT - 4 + 2 * lane);
    const bool out_lane = lane >= 2 && lane <= 29;
    const long long *Xl = (const long long *)X;
    auto rawx = [&](int64_t j) -> Pair {
      return (j >= 0 && j <= q.ny) ? ld_pair<V16>(Xl + j * q.pitch, c) : Pair{0ll, 0ll};
    };
    // GF is zero outside the interior, so any row inside the grid may be read
    auto rawg = [&](int64_t j) -> Pair {
      return (j >= 0 && j <= q.ny) ? ld_pair<V16>(GF + j * q.pitch, c) : Pair{0ll, 0ll};
    };
    Pair od_old = cvx(rawx(js - 1)), ev_new{0ll, 0ll};
    constexpr int PG = 1;
    Pair qe[PG], qo[PG], qge[PG], qgo[PG];  // raw X rows j, j+1 and GF rows j, j-1
#pragma unroll
    for (int t = 0; t < PG; ++t) {
      const int64_t j = js + 2 * t;
      const bool ok = j <= je;
      qe[t] = ok ? rawx(j) : Pair{0ll, 0ll};
      qo[t] = ok ? rawx(j + 1) : Pair{0ll, 0ll};
      qge[t] = ok ? rawg(j) : Pair{0ll, 0ll};
      qgo[t] = ok ? rawg(j - 1) : Pair{0ll, 0ll};
    }
    for (int64_t jb = js; jb <= je; jb += 2 * PG) {
#pragma unroll
      for (int t = 0; t < PG; ++t) {
        const int64_t j = jb + 2 * t;
        if (j > je) break;
        const Pair rc = cvx(qe[t]), rp = cvx(qo[t]);
        const Pair ge{qge[t].a >> dfr, qge[t].b >> dfr}, go{qgo[t].a >> dfr, qgo[t].b >> dfr};
        {
          const int64_t jn = j + 2 * PG;
          const bool ok = jn <= je;
          qe[t] = ok ? rawx(jn) : Pair{0ll, 0ll};
          qo[t] = ok ? rawx(jn + 1) : Pair{0ll, 0ll};
          qge[t] = ok ? rawg(jn) : Pair{0ll, 0ll};
          qgo[t] = ok ? rawg(jn - 1) : Pair{0ll, 0ll};
        }
        // even row j: colours 0 and 1 from the old rows j-1 and j+1
        Pair ue = rc;
        if (j >= 1 && j < q.ny) gs_pair(ue, Pair{od_old.a + rp.a, od_old.b + rp.b}, ge, c);
        // odd row j-1: colours 2 and 3 from the new rows j-2 and j
        if (j - 1 >= js + 1) {
          Pair uo = od_old;
          if (j - 1 < q.ny) gs_pair(uo, Pair{ev_new.a + ue.a, ev_new.b + ue.b}, go, c);
          put_pair<YF, V16>(q, Y, j - 1, c, out_lane, write_bnd, R, uo, hmax);
        }
        if (j < je || je == q.ny) put_pair<YF, V16>(q, Y, j, c, out_lane, write_bnd, R, ue, hmax);
        ev_new = ue;
        od_old = rp;
      }
    }
  }
  publish_bound(bnd, (sweep + 1) % 4, R, hmax, red);
}

// Two Gauss-Seidel sweeps in one pass over memory (temporal blocking).  A warp streams
// down its rows with four fronts, one step per even row j:
//   sweep 1, even row j    (colours 0, 1) from X rows j-1, j+1;
//   sweep 1, odd row j-1   (colours 2, 3) from sweep-1 even rows j-2, j;
//   sweep 2, even row j-2  (colours 0, 1) from sweep-1 odd rows j-3, j-1;
//   sweep 2, odd row j-3   (colours 2, 3) from sweep-2 even rows j-4, j-2;
// every input is the value the sequential colour order of two sweeps reads, and only
// sweep 2 is stored.  One sweep consumes four columns of the window per side (the
// shuffles of the two colour steps of each row), so of the 64 staged columns the 48 of
// lanes 4..27 hold sweep-2 values.  A chunk [js, je] starts its fronts at row js - 2 and
// runs them to je + 2, so that it can finish sweep 2 on its own rows (even js .. je - 2,
// odd js + 1 .. je - 1, and je when it is the last row) without another chunk's values.
// Scale: one R for both sweeps.  A sweep adds at most 4 * 3/8 h^2 max|f| to max|u| (one
// term per colour), so two sweeps stay below 2 (max|u| + 4 * 3/8 h^2 max|f|) <= 2^R (the
// spare bit of sweep_R); the int64 sums keep six more bits of headroom.  In FP64 mode
// (bound unusable) the same fronts run on FP64 buffers with the single-sweep kernel's
// FP64 formula.
constexpr int GS2X2_OUT = 48;

template <bool FIX>
__device__ __forceinline__ void gs_pair_t(Pair &u, const Pair &V, const Pair &gv, const Cols &c, double g) {
  if (FIX) {
    gs_pair(u, V, gv, c);
    return;
  }
  const long long Tb = add<false>(V.b, u.b);
  const long long Tbl = __shfl_up_sync(0xffffffffu, Tb, 1);
  if (c.ina) {
    const double N = __longlong_as_double(add<false>(add<false>(Tbl, Tb), V.a));
    u.a = __double_as_longlong(fma(N, 0.125, g * __longlong_as_double(gv.a)));
  }
  const long long Ta = add<false>(V.a, u.a);
  const long long Tar = __shfl_down_sync(0xffffffffu, Ta, 1);
  if (c.inb) {
    const double N = __longlong_as_double(add<false>(add<false>(Ta, Tar), V.b));
    u.b = __double_as_longlong(fma(N, 0.125, g * __longlong_as_double(gv.b)));
  }
}

template <bool FIX, int XF, int YF, bool V16>
__device__ __forceinline__ void gs2x2_rows(const Geo &q, const void *X, void *Y, const long long *rhs_arr,
                                           const Cols &c, int64_t js, int64_t je, int lane, const InScale<XF> &cvx,
                                           int dfr, double g, int R, bool write_bnd, unsigned &hmax) {
  const bool out_lane = lane >= 4 && lane <= 27;
  const long long *Xl = (const long long *)X;
  auto rawx = [&](int64_t j) -> Pair {
    return (j >= 0 && j <= q.ny) ? ld_pair<V16>(Xl + j * q.pitch, c) : Pair{0ll, 0ll};
  };
  // interior rows only: GF is zero elsewhere, and f off the interior is never used
  auto rawg = [&](int64_t j) -> Pair {
    return (j >= 1 && j < q.ny) ? ld_pair<V16>(rhs_arr + j * q.pitch, c) : Pair{0ll, 0ll};
  };
  auto in = [&](const Pair &p) -> Pair { return FIX ? cvx(p) : p; };
  auto rhs = [&](const Pair &p) -> Pair { return FIX ? Pair{p.a >> dfr, p.b >> dfr} : p; };
  auto vsum = [&](const Pair &x, const Pair &y) -> Pair { return Pair{add<FIX>(x.a, y.a), add<FIX>(x.b, y.b)}; };
  const Pair zero{0ll, 0ll};
  // carried from the step of row j - 2: X odd row j - 1; sweep-1 even row j - 2 and odd
  // row j - 3; sweep-2 even row j - 4; the right-hand sides of rows j - 2 and j - 3
  Pair od_old = in(rawx(js - 3)), s1e_prev = zero, s1o_prev = zero, s2e_prev = zero;
  Pair ge_prev = zero, go_prev = zero;
  // raw X rows j, j + 1 and right-hand-side rows j, j - 1 of the next step
  Pair qe = rawx(js - 2), qo = rawx(js - 1), qge = rawg(js - 2), qgo = rawg(js - 3);
  for (int64_t j = js - 2; j <= je + 2; j += 2) {
    const Pair rc = in(qe), rp = in(qo), ge = rhs(qge), go = rhs(qgo);
    {
      const int64_t jn = j + 2;
      const bool ok = jn <= je + 2;  // warp-uniform
      qe = ok ? rawx(jn) : zero;
      qo = ok ? rawx(jn + 1) : zero;
      qge = ok ? rawg(jn) : zero;
      qgo = ok ? rawg(jn - 1) : zero;
    }
    Pair s1e = rc;
    if (j >= 1 && j < q.ny) gs_pair_t<FIX>(s1e, vsum(od_old, rp), ge, c, g);
    Pair s1o = od_old;
    if (j - 1 >= 1 && j - 1 < q.ny) gs_pair_t<FIX>(s1o, vsum(s1e_prev, s1e), go, c, g);
    Pair s2e = s1e_prev;
    if (j - 2 >= 1 && j - 2 < q.ny) gs_pair_t<FIX>(s2e, vsum(s1o_prev, s1o), ge_prev, c, g);
    Pair s2o = s1o_prev;
    if (j - 3 >= 1 && j - 3 < q.ny) gs_pair_t<FIX>(s2o, vsum(s2e_prev, s2e), go_prev, c, g);
    // FP64 mode: the buffers hold FP64 bits, stored as they are
    if (j - 3 >= js + 1 && j - 3 <= je - 1) put_pair<FIX ? YF : SF_FXP, V16>(q, Y, j - 3, c, out_lane, write_bnd, R, s2o, hmax);
    if (j - 2 >= js && (j - 2 < je || je == q.ny))
      put_pair<FIX ? YF : SF_FXP, V16>(q, Y, j - 2, c, out_lane, write_bnd, R, s2e, hmax);
    od_old = rp;
    s1e_prev = s1e;
    s1o_prev = s1o;
    s2e_prev = s2e;
    ge_prev = ge;
    go_prev = go;
  }
}

template <int XF, int YF, bool V16>
__global__ void __launch_bounds__(W2_THREADS, S2X2_MIN_CTAS) k_gs2_sweep2(Geo q, const void *__restrict__ X, void *__restrict__ Y,
                                                           const double *__restrict__ f,
                                                           const long long *__restrict__ GF, SweepBounds *bnd,
                                                           int sweep, int sweeps, double g, bool write_bnd, int rows) {
  __shared__ unsigned red[W2_THREADS / 32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * (W2_THREADS / 32) + wib;
  const Plan plan = make_plan(bnd, g, sweeps);
  const int R = sweep_R(bnd, sweep % 4, g);
  const int Rx = sweep > 0 ? sweep_R(bnd, (sweep + 3) % 4, g) : R;
  const int dx = XF == SF_FXP ? R - Rx : 0, df = R - plan.Rf;
  InScale<XF> cvx{1023 + R, dx > 0 ? (dx < 63 ? dx : 63) : 0, dx < 0 ? (-dx < 63 ? -dx : 63) : 0};
  const int dfr = df < 63 ? df : 63;
  if (blockIdx.x == 0 && threadIdx.x == 0) bnd->umax[(sweep + 2) % 4] = 0ull;
  const int64_t nseg = (q.nx + GS2X2_OUT) / GS2X2_OUT;
  const int64_t seg = gw % nseg, chunk = gw / nseg;
  const int64_t js = chunk * rows;  // even
  unsigned hmax = 0;
  if (js <= q.ny) {
    int64_t je = js + rows;
    if (je > q.ny) je = (q.ny & 1) ? q.ny + 1 : q.ny;
    const Cols c = make_cols(q, seg * GS2X2_OUT - 8 + 2 * lane);
    if (plan.fix)
      gs2x2_rows<true, XF, YF, V16>(q, X, Y, GF, c, js, je, lane, cvx, dfr, g, R, write_bnd, hmax);
    else  // FP64 buffers throughout the call
      gs2x2_rows<false, SF_F64, SF_F64, V16>(q, X, Y, (const long long *)f, c, js, je, lane, InScale<SF_F64>{}, 0,
                                              g, R, write_bnd, hmax);
  }
  if (plan.fix) publish_bound(bnd, (sweep + 1) % 4, R, hmax, red);
}

// Multi-sweep damped Jacobi in the same global-scale fixed point (0 < omega <= 1):
//   u' = u + omega (3/8 h^2 f + N/8 - u),
// with omega applied as an integer product: floor(D * Wq / 2^62), Wq = omega 2^62
// rounded, exact to one unit of the last fixed-point place.  |u'| <= max|u| +
// omega 3/8 h^2 max|f|, within the bound of sweep_bounds.cuh.  If the plan rules out
// fixed point, every sweep of the call runs the FP64-capable single-sweep path on FP64
// buffers.  Lane pairs as in the Gauss-Seidel sweep; one column of halo per side, so a
// warp produces the 60 columns of lanes 1..30.


constexpr int JAC2_OUT = 60;

template <int XF, int YF, bool V16>
__global__ void __launch_bounds__(W2_THREADS) k_jac2_sweep(Geo q, const void *__restrict__ X, void *__restrict__ Y,
                                                           const double *__restrict__ f,
                                                           const long long *__restrict__ GF, SweepBounds *bnd,
                                                           int sweep, int sweeps, double g, double omega,
                                                           long long Wq, bool write_bnd, int rows) {
  __shared__ unsigned red[W2_THREADS / 32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * (W2_THREADS / 32) + wib;
  const Plan plan = make_plan(bnd, g, sweeps);
  if (!plan.fix) {
    // FP64 buffers throughout: the single-sweep kernel's work units (30-column
    // segments), grid-stride
    Op2Args a{};
    a.q = q;
    a.u = (const double *)X;
    a.f = f;
    a.out = (double *)Y;
    a.c1 = omega * g;
    a.c2 = -omega * 0.375 / 3.0;
    const int64_t units = ops2_units(q, rows);
    for (int64_t w = gw; w < units; w += (int64_t)gridDim.x * (W2_THREADS / 32)) {
      Stream2 s;
      ops2_warp<O2_JACOBI, V16>(a, lane, w, s, rows);
    }
    return;
  }
  const int R = sweep_R(bnd, sweep % 4, g);
  const int Rx = sweep > 0 ? sweep_R(bnd, (sweep + 3) % 4, g) : R;
  const int dx = XF == SF_FXP ? R - Rx : 0, df = R - plan.Rf;
  InScale<XF> cvx{1023 + R, dx > 0 ? (dx < 63 ? dx : 63) : 0, dx < 0 ? (-dx < 63 ? -dx : 63) : 0};
  const int dfr = df < 63 ? df : 63;
  if (blockIdx.x == 0 && threadIdx.x == 0) bnd->umax[(sweep + 2) % 4] = 0ull;
  const Omega om(Wq);
  const int64_t nseg = (q.nx + JAC2_OUT) / JAC2_OUT;
  const int64_t seg = gw % nseg, chunk = gw / nseg;
  const int64_t js = chunk * rows;
  unsigned hmax = 0;
  if (js <= q.ny) {
    const int64_t je = js + rows < q.ny + 1 ? js + rows : q.ny + 1;
    const Cols c = make_cols(q, seg * JAC2_OUT - 2 + 2 * lane);
    const bool out_lane = lane >= 1 && lane <= 30;
    const long long *Xl = (const long long *)X;
    auto rawx = [&](int64_t j) -> Pair {
      return (j >= 0 && j <= q.ny) ? ld_pair<V16>(Xl + j * q.pitch, c) : Pair{0ll, 0ll};
    };
    auto rawg = [&](int64_t j) -> Pair {
      return (j >= 0 && j <= q.ny) ? ld_pair<V16>(GF + j * q.pitch, c) : Pair{0ll, 0ll};
    };
    Pair um = cvx(rawx(js - 1)), uc = cvx(rawx(js)), up = cvx(rawx(js + 1));
    constexpr int PQ = 2;
    Pair qx[PQ], qg[PQ];  // raw X row j + 2 and GF row j for the iteration j = jb + t
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
        const Pair rn = qx[t], gr = qg[t];
        qx[t] = j + 2 + PQ <= je ? rawx(j + 2 + PQ) : Pair{0ll, 0ll};
        qg[t] = j + PQ < je ? rawg(j + PQ) : Pair{0ll, 0ll};
        const Pair V{um.a + up.a, um.b + up.b};
        const Pair T{V.a + uc.a, V.b + uc.b};
        const long long Tbl = __shfl_up_sync(0xffffffffu, T.b, 1);
        const long long Tar = __shfl_down_sync(0xffffffffu, T.a, 1);
        Pair un = uc;  // Dirichlet values carried
        if (j >= 1 && j < q.ny) {
          if (c.ina) un.a = uc.a + om((gr.a >> dfr) + ((Tbl + T.b + V.a) >> 3) - uc.a);
          if (c.inb) un.b = uc.b + om((gr.b >> dfr) + ((T.a + Tar + V.b) >> 3) - uc.b);
        }
        put_pair<YF, V16>(q, Y, j, c, out_lane, write_bnd, R, un, hmax);
        um = uc;
        uc = up;
        up = cvx(rn);
      }
    }
  }
  publish_bound(bnd, (sweep + 1) % 4, R, hmax, red);
}


// Two damped Jacobi sweeps in one pass (temporal blocking): a warp streaming down its
// rows computes sweep 1 at row j and sweep 2 at row j - 1 from sweep 1's rows j - 2 ..
// j, held in registers; only sweep 2 is stored.  Sweep 1 is computed on the staged
// columns 1..62 and sweep 2 on 2..61 (the 60 output columns of lanes 1..30); a chunk
// of rows [js, je) computes sweep 1 on rows js - 1 .. je.  Every sweep-2 value is the
// one two separate sweeps would produce: both use the same fixed-point scale (the
// tracked bound covers the growth of two damped sweeps, at most 2 omega 3/8 h^2 max|f|),
// and in FP64 mode (bound unusable) the same formula as the single-sweep kernel.
template <bool FIX>
__device__ __forceinline__ Pair jac_row(const Pair &m, const Pair &c, const Pair &p, const Pair &rhs, bool jin,
                                        const Cols &cl, int dfr, const Omega &om, double c1, double c2) {
  const Pair V{add<FIX>(m.a, p.a), add<FIX>(m.b, p.b)};
  const Pair T{add<FIX>(V.a, c.a), add<FIX>(V.b, c.b)};
  const long long Tbl = __shfl_up_sync(0xffffffffu, T.b, 1);
  const long long Tar = __shfl_down_sync(0xffffffffu, T.a, 1);
  Pair un = c;  // Dirichlet values carried
  if (jin) {
    if (FIX) {
      if (cl.ina) un.a = c.a + om((rhs.a >> dfr) + ((Tbl + T.b + V.a) >> 3) - c.a);
      if (cl.inb) un.b = c.b + om((rhs.b >> dfr) + ((T.a + Tar + V.b) >> 3) - c.b);
    } else {
      auto upd = [&](long long u, long long N, long long f) {
        const double Td = fma(8.0, __longlong_as_double(u), -__longlong_as_double(N));
        return __double_as_longlong(fma(c2, Td, fma(c1, __longlong_as_double(f), __longlong_as_double(u))));
      };
      if (cl.ina) un.a = upd(c.a, add<false>(add<false>(Tbl, T.b), V.a), rhs.a);
      if (cl.inb) un.b = upd(c.b, add<false>(add<false>(T.a, Tar), V.b), rhs.b);
    }
  }
  return un;
}

template <bool FIX, int XF, int YF, bool V16>
__device__ __forceinline__ void jac2x2_rows(const Geo &q, const void *X, void *Y, const long long *rhs_arr,
                                            const Cols &c, int64_t js, int64_t je, int lane, const InScale<XF> &cvx,
                                            int dfr, const Omega &om, double c1, double c2, int R, bool write_bnd,
                                            unsigned &hmax) {
  const bool out_lane = lane >= 1 && lane <= 30;
  const long long *Xl = (const long long *)X;
  auto rawx = [&](int64_t j) -> Pair {
    return (j >= 0 && j <= q.ny) ? ld_pair<V16>(Xl + j * q.pitch, c) : Pair{0ll, 0ll};
  };
  auto rawg = [&](int64_t j) -> Pair {
    return (j >= 1 && j < q.ny) ? ld_pair<V16>(rhs_arr + j * q.pitch, c) : Pair{0ll, 0ll};
  };
  auto in = [&](const Pair &p) -> Pair { return FIX ? cvx(p) : p; };
  Pair xm = in(rawx(js - 2)), xc = in(rawx(js - 1)), xp = in(rawx(js));
  Pair s1m{0ll, 0ll}, s1c{0ll, 0ll};  // sweep-1 rows j1 - 2, j1 - 1
  Pair gprev{0ll, 0ll};               // rhs row j1 - 1
  constexpr int PQ = 1;
  Pair qx[PQ], qg[PQ];  // raw X row j1 + 2 and rhs row j1 for the iteration j1 = jb + t
#pragma unroll
  for (int t = 0; t < PQ; ++t) {
    qx[t] = rawx(js + 1 + t);
    qg[t] = rawg(js - 1 + t);
  }
  for (int64_t jb = js - 1; jb <= je; jb += PQ) {
#pragma unroll
    for (int t = 0; t < PQ; ++t) {
      const int64_t j1 = jb + t;
      if (j1 > je) break;  // warp-uniform
      const Pair rn = qx[t], g1 = qg[t];
      qx[t] = j1 + PQ <= je ? rawx(j1 + 2 + PQ) : Pair{0ll, 0ll};
      qg[t] = j1 + PQ <= je ? rawg(j1 + PQ) : Pair{0ll, 0ll};
      // sweep 1 at row j1 from X rows j1 - 1, j1, j1 + 1
      const Pair s1n = jac_row<FIX>(xm, xc, xp, g1, j1 >= 1 && j1 < q.ny, c, dfr, om, c1, c2);
      // sweep 2 at row j1 - 1 from sweep-1 rows j1 - 2, j1 - 1, j1
      const int64_t j2 = j1 - 1;
      if (j2 >= js && j2 < je) {
        const Pair s2 = jac_row<FIX>(s1m, s1c, s1n, gprev, j2 >= 1 && j2 < q.ny, c, dfr, om, c1, c2);
        // FP64 mode: the buffers hold FP64 bits, stored as they are
        put_pair<FIX ? YF : SF_FXP, V16>(q, Y, j2, c, out_lane, write_bnd, R, s2, hmax);
      }
      s1m = s1c;
      s1c = s1n;
      gprev = g1;
      xm = xc;
      xc = xp;
      xp = in(rn);
    }
  }
}

template <int XF, int YF, bool V16>
__global__ void __launch_bounds__(W2_THREADS, S2X2_MIN_CTAS) k_jac2_sweep2(Geo q, const void *__restrict__ X, void *__restrict__ Y,
                                                            const double *__restrict__ f,
                                                            const long long *__restrict__ GF, SweepBounds *bnd,
                                                            int sweep, int sweeps, double g, double omega,
                                                            long long Wq, bool write_bnd, int rows) {
  __shared__ unsigned red[W2_THREADS / 32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * (W2_THREADS / 32) + wib;
  const Plan plan = make_plan(bnd, g, sweeps);
  const int R = sweep_R(bnd, sweep % 4, g);
  const int Rx = sweep > 0 ? sweep_R(bnd, (sweep + 3) % 4, g) : R;
  const int dx = XF == SF_FXP ? R - Rx : 0, df = R - plan.Rf;
  InScale<XF> cvx{1023 + R, dx > 0 ? (dx < 63 ? dx : 63) : 0, dx < 0 ? (-dx < 63 ? -dx : 63) : 0};
  const int dfr = df < 63 ? df : 63;
  if (blockIdx.x == 0 && threadIdx.x == 0) bnd->umax[(sweep + 2) % 4] = 0ull;
  const Omega om(Wq);
  const double c1 = omega * g, c2 = -omega * 0.375 / 3.0;
  const int64_t nseg = (q.nx + JAC2_OUT) / JAC2_OUT;
  const int64_t seg = gw % nseg, chunk = gw / nseg;
  const int64_t js = chunk * rows;
  unsigned hmax = 0;
  if (js <= q.ny) {
    const int64_t je = js + rows < q.ny + 1 ? js + rows : q.ny + 1;
    const Cols c = make_cols(q, seg * JAC2_OUT - 2 + 2 * lane);
    if (plan.fix)
      jac2x2_rows<true, XF, YF, V16>(q, X, Y, GF, c, js, je, lane, cvx, dfr, om, c1, c2, R, write_bnd, hmax);
    else  // FP64 buffers throughout the call
      jac2x2_rows<false, SF_F64, SF_F64, V16>(q, X, Y, (const long long *)f, c, js, je, lane, InScale<SF_F64>{},
                                               0, om, c1, c2, R, write_bnd, hmax);
  }
  if (plan.fix) {
    publish_bound(bnd, (sweep + 1) % 4, R, hmax, red);
  }
}

}  // namespace

// Null counts as aligned (an absent array is never accessed).
static bool aligned16(const void *p) { return ((uintptr_t)p % 16) == 0; }

size_t ops2_reduce_bytes(const Geo &q) { return 16 + (size_t)ops2_blocks(q, W2_ROWS) * 2 * sizeof(double); }

// Rows per warp from a tuned shape: even, in [16, 4096]; `fallback` when none is set.
static int tuned_rows(int call, const Geo &q, int fallback) {
  const int r = tuned_chunk(tuning_lookup(call, q), fallback, 16, 4096);
  return r & ~1;
}

static cudaError_t launch_ops2(int op, const Op2Args &a, cudaStream_t s) {
  const unsigned nb = ops2_blocks(a.q, a.rows);
  // 16-byte row pairs: even pitch and 16-byte aligned u, f and output
  const bool v16 = a.q.pitch % 2 == 0 && aligned16(a.u) && aligned16(a.f) && aligned16(a.out);
  if (v16) {
    switch (op) {
      case O2_APPLY: k_ops2<O2_APPLY, true><<<nb, W2_THREADS, 0, s>>>(a); break;
      case O2_JACOBI: k_ops2<O2_JACOBI, true><<<nb, W2_THREADS, 0, s>>>(a); break;
      case O2_RESIDUAL: k_ops2<O2_RESIDUAL, true><<<nb, W2_THREADS, 0, s>>>(a); break;
      default: k_ops2<O2_ELEMENTWISE, true><<<nb, W2_THREADS, 0, s>>>(a); break;
    }
  } else {
    switch (op) {
      case O2_APPLY: k_ops2<O2_APPLY, false><<<nb, W2_THREADS, 0, s>>>(a); break;
      case O2_JACOBI: k_ops2<O2_JACOBI, false><<<nb, W2_THREADS, 0, s>>>(a); break;
      case O2_RESIDUAL: k_ops2<O2_RESIDUAL, false><<<nb, W2_THREADS, 0, s>>>(a); break;
      default: k_ops2<O2_ELEMENTWISE, false><<<nb, W2_THREADS, 0, s>>>(a); break;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_apply_fx2(const Geo &q, const double *u, double *y, bool elementwise, cudaStream_t s) {
  Op2Args a{};
  a.q = q;
  a.u = u;
  a.out = y;
  a.c1 = elementwise ? 1.0 / (6.0 * q.h * q.h) : 1.0 / (3.0 * q.h * q.h);
  a.rows = tuned_rows(elementwise ? STENCIL_CALL_APPLY_ELEMENTWISE : STENCIL_CALL_APPLY_STENCIL, q, W2_ROWS);
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
  a.rows = W2_ROWS;
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
  a.rows = W2_ROWS;
  return launch_ops2(O2_RESIDUAL, a, s);
}

// work: 3 arrays of u's span (8 bytes per element): two int64 ping-pong buffers and
// GF; bounds: gs_fx_bounds_bytes() bytes.  The result always ends in u, whose boundary
// values are never written.
cudaError_t launch_gs_sweeps_fx2(const Geo &q, double *u, const double *f, int sweeps, double *work, void *bounds,
                                 cudaStream_t s) {
  const double g = 0.375 * q.h * q.h;
  const Tuning tune = tuning_lookup(STENCIL_CALL_SMOOTH_COLOURED, q);
  const int rows = tuned_chunk(tune, S2_ROWS, 16, 4096) & ~1;
  const bool depth1 = tune.depth == 1;  // a tuned shape may ask for one sweep per pass
  const int64_t span = span_elems(q);
  cudaError_t e;
  if (sweeps == 1) {
    const int64_t nchunk = (q.ny + S2_ROWS) / S2_ROWS;
    const int64_t nseg = (q.nx + 24) / 24;
    const unsigned nb = (unsigned)((nseg * nchunk + W2_THREADS / 32 - 1) / (W2_THREADS / 32));
    k_gs2_fused<<<nb, W2_THREADS, 0, s>>>(q, u, work, f, g);
    e = cudaGetLastError();
    return e ? e : cudaMemcpyAsync(u, work, (size_t)span * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  const int64_t nchunk = (q.ny + rows) / rows;
  const int64_t nseg = (q.nx + GS2_OUT) / GS2_OUT, nseg2 = (q.nx + GS2X2_OUT) / GS2X2_OUT;
  const unsigned nb = (unsigned)((nseg * nchunk + W2_THREADS / 32 - 1) / (W2_THREADS / 32));
  const unsigned nb2 = (unsigned)((nseg2 * nchunk + W2_THREADS / 32 - 1) / (W2_THREADS / 32));
  void *A = work, *B = work + span;
  long long *GF = (long long *)(work + 2 * span);
  SweepBounds *bnd = (SweepBounds *)bounds;
  e = launch_gs_prepass(q, 2, u, f, GF, bounds, sweeps, s);
  // 16-byte row pairs need an even pitch and 16-byte aligned bases (u and work; the
  // buffers inside work then follow, span being even); the two-sweep kernel also reads
  // f in pairs when the bound rules out fixed point
  const bool v16 = q.pitch % 2 == 0 && aligned16(u) && aligned16(work);
  const bool v16f = v16 && aligned16(f);
  // two sweeps per launch (temporal blocking), a single-sweep launch for an odd rest
  const void *X = u;
  int done = 0;
  for (int it = 0; done < sweeps && !e; ++it) {
    // a two-sweep launch reads X and writes Y, so it is never both the first (X = u) and
    // the last (Y = u) launch: two sweeps in all go as two single-sweep launches
    const bool two = !depth1 && sweeps - done >= 2 && sweeps != 2;
    const bool first = done == 0, last = done + (two ? 2 : 1) == sweeps;
    void *Y = last ? (void *)u : (it % 2 == 0 ? A : B);
    // the caller's u (last launch): its Dirichlet values were never overwritten, leave them
    const bool wb = !last;
#define GS2_LAUNCH(KER, NB, XF_, YF_, V) \
  KER<XF_, YF_, V><<<NB, W2_THREADS, 0, s>>>(q, X, Y, f, GF, bnd, it, sweeps, g, wb, rows)
#define GS2_PICK(KER, NB, V)                   \
  do {                                         \
    if (first)                                 \
      GS2_LAUNCH(KER, NB, SF_F64, SF_FXP, V);  \
    else if (!last)                            \
      GS2_LAUNCH(KER, NB, SF_FXP, SF_FXP, V);  \
    else                                       \
      GS2_LAUNCH(KER, NB, SF_FXP, SF_F64, V);  \
  } while (0)
    if (two) {
      if (v16f)
        GS2_PICK(k_gs2_sweep2, nb2, true);
      else
        GS2_PICK(k_gs2_sweep2, nb2, false);
    } else {
      if (v16)
        GS2_PICK(k_gs2_sweep, nb, true);
      else
        GS2_PICK(k_gs2_sweep, nb, false);
    }
#undef GS2_PICK
#undef GS2_LAUNCH
    e = cudaGetLastError();
    X = Y;
    done += two ? 2 : 1;
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
  const Tuning tune = tuning_lookup(STENCIL_CALL_SMOOTH_JACOBI, q);
  const int rows = tuned_chunk(tune, S2_ROWS, 16, 4096) & ~1;
  const bool depth1 = tune.depth == 1;
  const int64_t nseg = (q.nx + JAC2_OUT) / JAC2_OUT;
  const int64_t nchunk = (q.ny + rows) / rows;
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
  // 16-byte row pairs: even pitch and 16-byte aligned u, f (read by the FP64 path),
  // A and scratch (the buffers inside scratch then follow, span being even)
  const bool v16 = q.pitch % 2 == 0 && aligned16(u) && aligned16(f) && aligned16(A) && aligned16(scratch);
  // two sweeps per launch (temporal blocking), a single-sweep launch for an odd rest
  const void *X = u;
  int done = 0;
  for (int it = 0; done < sweeps && !e; ++it) {
    // a fused launch reads X and writes Y, so it is never both the first (X = u) and the
    // last (Y = u) launch: two sweeps in all go as two single-sweep launches
    const bool two = !depth1 && sweeps - done >= 2 && sweeps != 2;
    const bool first = done == 0, last = done + (two ? 2 : 1) == sweeps;
    void *Y = last ? (void *)u : (it % 2 == 0 ? (void *)A : B);
    const bool wb = !last;  // the caller's u keeps its Dirichlet values
#define JAC2_LAUNCH(KER, XF_, YF_, V)                                                                   \
  KER<XF_, YF_, V><<<nb, W2_THREADS, 0, s>>>(q, X, Y, f, GF, bnd, it, sweeps, g, omega, Wq, wb, rows)
#define JAC2_PICK(KER, V)                                   \
  do {                                                      \
    if (first)                                              \
      JAC2_LAUNCH(KER, SF_F64, SF_FXP, V);                  \
    else if (!last)                                         \
      JAC2_LAUNCH(KER, SF_FXP, SF_FXP, V);                  \
    else                                                    \
      JAC2_LAUNCH(KER, SF_FXP, SF_F64, V);                  \
  } while (0)
    if (two) {
      if (v16)
        JAC2_PICK(k_jac2_sweep2, true);
      else
        JAC2_PICK(k_jac2_sweep2, false);
    } else {
      if (v16)
        JAC2_PICK(k_jac2_sweep, true);
      else
        JAC2_PICK(k_jac2_sweep, false);
    }
#undef JAC2_PICK
#undef JAC2_LAUNCH
    e = cudaGetLastError();
    X = Y;
    done += two ? 2 : 1;
  }
  return e;
}

}  // namespace stencil
