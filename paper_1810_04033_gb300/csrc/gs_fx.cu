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
// Two kernels implement the half sweep: k_gs_half_t (further below) stages the planes by
// TMA and works on column pairs; it is used whenever the arrays allow it (16-byte
// aligned, even pitch).  k_gs_half_sweep, described next, stages through registers and
// takes the remaining cases (and the single-sweep FP64 -> FP64 call).
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
#include "sweep_bounds.cuh"
#include "tma.cuh"

namespace stencil {
namespace {

constexpr int GS_TX = 58, GS_TY = 30;        // output tile
constexpr int GS_SW = 64;                    // staged columns (62 used)
constexpr int GS_SH = 36;                    // staged rows (34 used, 2 zero pad rows)
constexpr int GS_THREADS = 256;
constexpr int GS_CZ = 16;                    // centre planes per CTA (at most)
constexpr int GS_NUP = GS_SH * GS_SW / GS_THREADS;             // 9 values / thread
constexpr int GS_NCE = (GS_SH / 2 * GS_SW + GS_THREADS - 1) / GS_THREADS;  // 5 (odd rows)
constexpr size_t GS_PLANE = (size_t)GS_SH * GS_SW;
constexpr size_t GS_SMEM = 3 * GS_PLANE * sizeof(long long);

enum { F64 = 0, FXP = 1 };  // storage format of an array: FP64, or int64 fixed point

struct Ctx {
  Geo q;
  int x0, y0;        // tile origin (vertex indices)
  int R;             // scale of this sweep: values are multiples of 2^(R - 52), |v| < 2^R
  int dx, dn, df;    // right shifts taking X, N and GF to this sweep's scale
  double g;          // 3/8 h^2
  int nx, ny, pitch;
  bool write_bnd;    // write Dirichlet copies into Y (false when Y is the caller's u)
};

__device__ __forceinline__ long long shr(long long v, int d) { return shr_any(v, d); }

// Raw 64-bit load (FP64 bits or int64) of element `off` of plane pointer p.
__device__ __forceinline__ long long ld64(const void *p, int off) {
  return ((const long long *)p)[off];
}

// Convert a raw staged value of format SF into this sweep's representation.
template <bool FIXA, int SF>
__device__ __forceinline__ long long to_rep(long long raw, int rb, int d) {
  if (!FIXA) return raw;                                    // FP64 arithmetic: keep the bits
  if (SF == F64) return fx::to_fixed(__longlong_as_double(raw), rb);
  return d ? shr(raw, d) : raw;
}

template <bool FIXA>
__device__ __forceinline__ long long add(long long a, long long b) {
  if (FIXA) return a + b;
  return __double_as_longlong(__longlong_as_double(a) + __longlong_as_double(b));
}

template <bool INNER>
__device__ __forceinline__ bool staged_at(const Ctx &c, int r, int col, int &off) {
  const int x = c.x0 - 2 + col, j = c.y0 - 2 + r;
  off = j * c.pitch + x;
  if (INNER) return col < GS_TX + 4 && r < GS_TY + 4;
  return col < GS_TX + 4 && r < GS_TY + 4 && x >= 0 && x <= c.nx && j >= 0 && j <= c.ny;
}

// Prefetch (raw 64-bit) of one centre plane's odd rows and one full neighbour plane.
template <bool INNER>
__device__ __forceinline__ void prefetch(const Ctx &c, const void *cplane, const void *uplane,
                                         long long (&pc)[GS_NCE], long long (&pu)[GS_NUP]) {
#pragma unroll
  for (int k = 0; k < GS_NCE; ++k) {
    const int idx = threadIdx.x + k * GS_THREADS;
    const int r = 2 * (idx >> 6) + 1, col = idx & 63;
    int off;
    const bool ok = idx < GS_SH / 2 * GS_SW && cplane && staged_at<INNER>(c, r, col, off);
    pc[k] = ok ? ld64(cplane, off) : 0ll;
  }
#pragma unroll
  for (int k = 0; k < GS_NUP; ++k) {
    const int idx = threadIdx.x + k * GS_THREADS;
    const int r = idx >> 6, col = idx & 63;
    int off;
    const bool ok = uplane && staged_at<INNER>(c, r, col, off);
    pu[k] = ok ? ld64(uplane, off) : 0ll;
  }
}

template <bool FIXA, int CF, int UF>
__device__ __forceinline__ void commit(const Ctx &c, const long long (&pc)[GS_NCE],
                                       const long long (&pu)[GS_NUP], long long *ce, long long *up,
                                       int dup) {
  const int rb = 1023 + c.R;
#pragma unroll
  for (int k = 0; k < GS_NCE; ++k) {
    const int idx = threadIdx.x + k * GS_THREADS;
    if (idx < GS_SH / 2 * GS_SW)
      ce[(2 * (idx >> 6) + 1) * GS_SW + (idx & 63)] = to_rep<FIXA, CF>(pc[k], rb, c.dx);
  }
#pragma unroll
  for (int k = 0; k < GS_NUP; ++k) up[threadIdx.x + k * GS_THREADS] = to_rep<FIXA, UF>(pu[k], rb, dup);
}

// Right-hand side values for the two phases of one centre plane (4 rows each): GF
// (int64, 3/8 h^2 f in fixed point) in fixed arithmetic, f itself otherwise.
template <bool INNER>
__device__ __forceinline__ void prefetch_f(const Ctx &c, const void *fplane, long long (&fv)[8]) {
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
      fv[4 * ph + k] = ok ? ld64(fplane, j * c.pitch + x) : 0ll;
    }
  }
}

// One phase on the staged centre plane.  WHICH = 1: rows of parity 0 on the tile + 1
// (results also written back into the centre plane); WHICH = 2: rows of parity 1 on
// the tile.  A warp walks 4 rows of one 32-column segment, carrying the column sums of
// the shared rows from one row to the next.
template <bool FIXA, int XF, int YF, bool INNER, int WHICH>
__device__ __forceinline__ void phase(const Ctx &c, long long *ce, const long long *lo,
                                      const long long *up, const void *xplane, void *yplane,
                                      const long long (&fv)[8], long long &vmax) {
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
  long long Dm = add<FIXA>(lc[(r0 - 1) * GS_SW], uc[(r0 - 1) * GS_SW]);
  long long Cm = cc[(r0 - 1) * GS_SW];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = r0 + 2 * k;
    const long long Dp = add<FIXA>(lc[(r + 1) * GS_SW], uc[(r + 1) * GS_SW]);
    const long long Cp = cc[(r + 1) * GS_SW];
    const long long W = add<FIXA>(lc[r * GS_SW], uc[r * GS_SW]);
    const long long V = add<FIXA>(Cm, Cp);
    const long long Q = add<FIXA>(Dm, Dp);
    const long long VW = add<FIXA>(V, W);
    const long long P = add<FIXA>(add<FIXA>(VW, VW), Q);
    const long long Pm = __shfl_up_sync(0xffffffffu, P, 1);
    const long long Pp = __shfl_down_sync(0xffffffffu, P, 1);
    Dm = Dp;
    Cm = Cp;
    const int j = c.y0 - 2 + r;
    const bool row_ok = WHICH == 1 ? true : r <= GS_TY + 1;  // phase 2: last group has 3 rows
    if (!lane_out || !row_ok) continue;
    const bool in_grid = x_in && (INNER || (j >= 0 && j <= c.ny));
    if (!in_grid) continue;
    const bool inner = x_inner && (INNER || (j >= 1 && j < c.ny));
    const int off = j * c.pitch + x;
    const bool core = col_core && (WHICH == 2 || r < GS_TY + 2);
    long long rep;  // new value in this sweep's representation
    if (inner) {
      const long long S = add<FIXA>(add<FIXA>(Pm, Pp), add<FIXA>(Q, Q));  // 2E + C
      if (FIXA)
        rep = (fv[(WHICH - 1) * 4 + k] >> c.df) + (S >> 5);
      else
        rep = __double_as_longlong(fma(__longlong_as_double(S), 0.03125,
                                       c.g * __longlong_as_double(fv[(WHICH - 1) * 4 + k])));
    } else {
      // Dirichlet value, carried through
      rep = to_rep<FIXA, XF>(ld64(xplane, off), 1023 + c.R, c.dx);
      if (!c.write_bnd) {
        if (WHICH == 1) cc[r * GS_SW] = rep;
        continue;
      }
    }
    if (WHICH == 1) cc[r * GS_SW] = rep;
    if (core) {
      if (YF == FXP && FIXA) {
        ((long long *)yplane)[off] = rep;
      } else if (FIXA) {
        ((double *)yplane)[off] = inner ? fx::to_double_cvt(rep, c.R - fx::FRAC) : __longlong_as_double(ld64(xplane, off));
      } else {
        ((long long *)yplane)[off] = rep;  // FP64 bits
      }
      const long long a = FIXA ? (rep < 0 ? -rep : rep) : (long long)fx::abs_bits(__longlong_as_double(rep));
      vmax = a > vmax ? a : vmax;
    }
  }
}

template <bool FIXA, int XF, int NF, int YF, bool INNER>
__device__ void run_half(Ctx &c, int pz, int i0, int i1, const void *X, const void *N, void *Y,
                         const void *F, long long *smem, long long &vmax) {
  const Geo &q = c.q;
  const int64_t P = q.plane;
  auto slot = [&](int i) -> long long * { return smem + i * GS_PLANE; };
  int lo = 0, ce = 1, up = 2;
  long long pc[GS_NCE], pu[GS_NUP], fv[8];
  const char *Xc = (const char *)X, *Nc = (const char *)N, *Fc = (const char *)F;
  char *Yc = (char *)Y;
  {
    const int64_t z = pz + 2 * (int64_t)i0;
    long long dummy[GS_NCE];
    prefetch<INNER>(c, nullptr, z >= 1 ? Nc + (z - 1) * P * 8 : nullptr, dummy, pu);
    commit<FIXA, XF, NF>(c, dummy, pu, slot(ce), slot(lo), c.dn);
    const bool zin = z >= 1 && z <= q.nz - 1;
    prefetch<INNER>(c, zin ? Xc + z * P * 8 : nullptr, z + 1 <= q.nz ? Nc + (z + 1) * P * 8 : nullptr, pc, pu);
    prefetch_f<INNER>(c, zin ? Fc + z * P * 8 : nullptr, fv);
  }
  for (int i = i0; i < i1; ++i) {
    const int64_t z = pz + 2 * (int64_t)i;
    const bool zin = z >= 1 && z <= q.nz - 1;
    commit<FIXA, XF, NF>(c, pc, pu, slot(ce), slot(up), c.dn);
    long long fcur[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) fcur[k] = fv[k];
    __syncthreads();
    if (i + 1 < i1) {  // next centre plane z + 2 and its upper neighbour z + 3
      const bool zn = z + 2 >= 1 && z + 2 <= q.nz - 1;
      prefetch<INNER>(c, zn ? Xc + (z + 2) * P * 8 : nullptr, z + 3 <= q.nz ? Nc + (z + 3) * P * 8 : nullptr,
                      pc, pu);
      prefetch_f<INNER>(c, zn ? Fc + (z + 2) * P * 8 : nullptr, fv);
    }
    const void *xp = Xc + z * P * 8;
    void *yp = Yc + z * P * 8;
    if (zin) {
      phase<FIXA, XF, YF, INNER, 1>(c, slot(ce), slot(lo), slot(up), xp, yp, fcur, vmax);
      __syncthreads();
      phase<FIXA, XF, YF, INNER, 2>(c, slot(ce), slot(lo), slot(up), xp, yp, fcur, vmax);
    } else if (c.write_bnd) {
      // Dirichlet plane: carry the tile through
      for (int idx = threadIdx.x; idx < GS_TX * GS_TY; idx += GS_THREADS) {
        const int x = c.x0 + idx % GS_TX, j = c.y0 + idx / GS_TX;
        if (x > c.nx || j > c.ny) continue;
        const int off = j * c.pitch + x;
        const long long raw = ld64(xp, off);
        long long out, a;
        if (FIXA && YF == FXP) {
          out = to_rep<FIXA, XF>(raw, 1023 + c.R, c.dx);
          a = out < 0 ? -out : out;
        } else if (FIXA) {  // FP64 output of an FP64 or fixed input
          out = XF == F64 ? raw : __double_as_longlong(fx::to_double(shr(raw, c.dx), c.R - fx::FRAC));
          a = XF == F64 ? to_rep<true, F64>(raw, 1023 + c.R, 0) : shr(raw, c.dx);
          a = a < 0 ? -a : a;
        } else {
          out = raw;
          a = (long long)fx::abs_bits(__longlong_as_double(raw));
        }
        ((long long *)yp)[off] = out;
        vmax = a > vmax ? a : vmax;
      }
    }
    __syncthreads();
    // the upper neighbour becomes the next centre plane's lower neighbour
    const int t = lo;
    lo = up;
    up = t;
  }
}

template <int XF, int NF, int YF>
__global__ void __launch_bounds__(GS_THREADS, 2)
    k_gs_half_sweep(Geo q, int pz, const void *X, const void *N, void *Y, const double *f, const long long *GF,
                    SweepBounds *bnd, int sweep, int sweeps, double g, int cz,
                    bool write_bnd) {
  extern __shared__ long long smem[];
  __shared__ long long red[GS_THREADS / 32];
  Ctx c;
  c.q = q;
  c.x0 = (int)blockIdx.x * GS_TX;
  c.y0 = (int)blockIdx.y * GS_TY;
  c.g = g;
  c.nx = (int)q.nx;
  c.ny = (int)q.ny;
  c.pitch = (int)q.pitch;
  c.write_bnd = write_bnd;
  const Plan plan = make_plan(bnd, g, sweeps);
  const int rd = sweep % 4, wr = (sweep + 1) % 4, cl = (sweep + 2) % 4;
  c.R = sweep_R(bnd, rd, g);
  const int Rx = sweep > 0 ? sweep_R(bnd, (sweep + 3) % 4, g) : c.R;  // scale of the previous sweep
  c.dx = XF == FXP ? c.R - Rx : 0;
  c.dn = NF == FXP ? (pz == 0 ? c.dx : 0) : 0;  // odd launch: N is this sweep's output
  // R >= Rf (the sweep's bound includes 4 (3/8) h^2 max|f|): GF needs a right shift,
  // clamped at 63 (which leaves 0 or -1, below one unit of the last place)
  c.df = min(c.R - plan.Rf, 63);
  if (pz == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0)
    bnd->umax[cl] = 0ull;  // to be accumulated by sweep s + 1

  const int ncentre = q.nz >= pz ? (int)((q.nz - pz) / 2 + 1) : 0;
  const int i0 = (int)blockIdx.z * cz;
  const int i1 = i0 + cz < ncentre ? i0 + cz : ncentre;
  const bool inner = c.x0 >= 2 && c.x0 + GS_TX + 1 <= c.nx && c.y0 >= 2 && c.y0 + GS_TY + 1 <= c.ny;
  long long vmax = 0;
  if (plan.fix) {
    if (inner)
      run_half<true, XF, NF, YF, true>(c, pz, i0, i1, X, N, Y, GF, smem, vmax);
    else
      run_half<true, XF, NF, YF, false>(c, pz, i0, i1, X, N, Y, GF, smem, vmax);
  } else {
    run_half<false, F64, F64, F64, false>(c, pz, i0, i1, X, N, Y, f, smem, vmax);
  }
  // block max of |new values| -> FP64 bits -> the next sweep's bound
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long w = __shfl_xor_sync(0xffffffffu, vmax, o);
    vmax = w > vmax ? w : vmax;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = vmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long m = 0;
    for (int w = 0; w < GS_THREADS / 32; ++w) m = red[w] > m ? red[w] : m;
    const unsigned long long mb =
        plan.fix ? fx::abs_bits(fx::to_double(m, c.R - fx::FRAC) * (1.0 + 0x1p-50)) : (unsigned long long)m;
    atomicMax(&bnd->umax[wr], mb);
  }
}

// ------------------------------------------------------------ TMA-staged form
// The same half sweep with the planes brought into shared memory by TMA
// (cp.async.bulk.tensor, one mbarrier per slot, bounded waits): five plane slots hold
// the neighbour planes z-1 and z+1 (from N), the centre plane z (from X) and, in
// flight, the next centre plane's two new planes, issued one centre plane ahead.  A
// staged box is 64 x 34 vertices from (x0 - 2, y0 - 2), x0 even, so staged column c is
// x0 - 2 + c and row r is y0 - 2 + r; lane l works on the column pair 2l, 2l + 1.
// Phase 1 (even rows, the tile grown by one vertex) writes its results into the staged
// centre plane, whose other values are the old ones (Dirichlet vertices stay as they
// are); phase 2 (odd rows, the tile) reads them.  Staged int64 planes already at this
// sweep's scale are used as they arrive; FP64 planes (first sweep) or a scale change
// are converted in place.  Used when X, N and Y are 16-byte aligned with an even pitch
// and the result is fixed point or the Dirichlet values are not written (an exact FP64
// copy of them stays with k_gs_half_sweep).  A wait that runs out sets
// g_gs_tma_error and the CTA leaves (its part of the sweep is then missing).
constexpr int GT_W = 64, GT_H = 34;          // staged box
constexpr int GT_TX = 60, GT_TY = 30;        // output tile
constexpr int GT_THREADS = 256;
constexpr int GT_SLOT = GT_W * GT_H;         // elements per slot (17408 bytes)
constexpr int GT_NSLOT = 5;
constexpr size_t GT_SMEM = (size_t)GT_NSLOT * GT_SLOT * sizeof(long long) + 128;
constexpr unsigned GT_WAIT = 1u << 22;
__device__ unsigned g_gs_tma_error = 0;

struct LP {
  long long a, b;
};

template <bool FIXA>
__device__ __forceinline__ LP addp(const LP &x, const LP &y) {
  return LP{add<FIXA>(x.a, y.a), add<FIXA>(x.b, y.b)};
}

__device__ __forceinline__ LP ldsp(const long long *p) {
  const longlong2 v = *(const longlong2 *)p;
  return LP{v.x, v.y};
}

// Right-hand side pair (GF in fixed arithmetic, f otherwise) of row j at columns xa,
// xa + 1 for an interior row; zeros where the columns leave the grid.
template <bool INNER>
__device__ __forceinline__ LP ld_rhs(const Ctx &c, const void *fplane, int j, int xa) {
  LP p{0ll, 0ll};
  if (!fplane || j < 1 || j >= c.ny) return p;
  const long long *row = (const long long *)fplane + (int64_t)j * c.pitch;
  if (INNER || (xa >= 0 && xa + 1 <= c.nx)) {
    const longlong2 v = *(const longlong2 *)(row + xa);
    p.a = v.x;
    p.b = v.y;
  } else if (xa >= 0 && xa <= c.nx) {
    p.a = row[xa];
  }
  return p;
}

// One phase on the staged centre plane for the pair rows r0 and r0 + 2 of this warp.
// WHICH = 1: even rows 2 + 4w, 4 + 4w on staged columns 1..62 (results also written
// back into the centre plane); WHICH = 2: odd rows 3 + 4w, 5 + 4w (up to 31) on
// columns 2..61.  Y receives the core (columns 2..61, rows 2..31) inside the grid.
template <bool FIXA, int YF, bool INNER, int WHICH>
__device__ __forceinline__ void phase_t(const Ctx &c, long long *ce, const long long *lo, const long long *up,
                                        void *yplane, const LP (&fv)[2], long long &vmax) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col = 2 * lane;
  const int r0 = (WHICH == 1 ? 2 : 3) + 4 * warp;
  const int xa = c.x0 - 2 + col;
  // columns this phase computes: WHICH 1: 1..62, WHICH 2: 2..61
  const bool va = WHICH == 1 ? lane >= 1 : (lane >= 1 && lane <= 30);
  const bool vb = WHICH == 1 ? lane <= 30 : (lane >= 1 && lane <= 30);
  const bool core = lane >= 1 && lane <= 30;
  const bool xa_in = INNER || (xa >= 1 && xa < c.nx), xb_in = INNER || (xa + 1 >= 1 && xa + 1 < c.nx);
  const bool xa_ok = INNER || (xa >= 0 && xa <= c.nx), xb_ok = INNER || (xa + 1 >= 0 && xa + 1 <= c.nx);
  const long long *lc = lo + col, *uc = up + col;
  long long *cc = ce + col;
  LP Dm = addp<FIXA>(ldsp(lc + (r0 - 1) * GT_W), ldsp(uc + (r0 - 1) * GT_W));
  LP Cm = ldsp(cc + (r0 - 1) * GT_W);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int r = r0 + 2 * k;
    if (WHICH == 2 && r > 31) break;  // warp-uniform
    const LP Dp = addp<FIXA>(ldsp(lc + (r + 1) * GT_W), ldsp(uc + (r + 1) * GT_W));
    const LP Cp = ldsp(cc + (r + 1) * GT_W);
    const LP W = addp<FIXA>(ldsp(lc + r * GT_W), ldsp(uc + r * GT_W));
    const LP V = addp<FIXA>(Cm, Cp);
    const LP Q = addp<FIXA>(Dm, Dp);
    const LP VW = addp<FIXA>(V, W);
    const LP P = addp<FIXA>(addp<FIXA>(VW, VW), Q);
    const long long Pl = __shfl_up_sync(0xffffffffu, P.b, 1);
    const long long Pr = __shfl_down_sync(0xffffffffu, P.a, 1);
    Dm = Dp;
    Cm = Cp;
    const int j = c.y0 - 2 + r;
    const bool jin = INNER || (j >= 1 && j < c.ny);
    const bool ja = va && xa_in && jin, jb = vb && xb_in && jin;  // updated vertices
    const LP old = ldsp(cc + r * GT_W);
    LP nw = old;
    const long long Sa = add<FIXA>(add<FIXA>(Pl, P.b), add<FIXA>(Q.a, Q.a));  // 2E + C
    const long long Sb = add<FIXA>(add<FIXA>(P.a, Pr), add<FIXA>(Q.b, Q.b));
    if (FIXA) {
      if (ja) nw.a = (fv[k].a >> c.df) + (Sa >> 5);
      if (jb) nw.b = (fv[k].b >> c.df) + (Sb >> 5);
    } else {
      if (ja) nw.a = __double_as_longlong(fma(__longlong_as_double(Sa), 0.03125, c.g * __longlong_as_double(fv[k].a)));
      if (jb) nw.b = __double_as_longlong(fma(__longlong_as_double(Sb), 0.03125, c.g * __longlong_as_double(fv[k].b)));
    }
    if (WHICH == 1) *(longlong2 *)(cc + r * GT_W) = make_longlong2(nw.a, nw.b);
    // Y: core rows 2..31 inside the grid; Dirichlet copies only if write_bnd
    const bool jok = INNER || (j >= 0 && j <= c.ny);
    const bool rcore = r >= 2 && r <= 31;
    const bool wa = core && rcore && jok && xa_ok && (ja || c.write_bnd);
    const bool wb = core && rcore && jok && xb_ok && (jb || c.write_bnd);
    if (INNER && FIXA && YF == FXP) {
      // inside the grid both columns of a core lane are updated and written
      if (core && rcore) {
        *(longlong2 *)((long long *)yplane + (int64_t)j * c.pitch + xa) = make_longlong2(nw.a, nw.b);
        const long long ma = nw.a < 0 ? -nw.a : nw.a, mb = nw.b < 0 ? -nw.b : nw.b;
        vmax = max(vmax, max(ma, mb));
      }
    } else if (wa || wb) {
      long long ya = nw.a, yb = nw.b;
      if (FIXA && YF == F64) {  // last sweep: only updated vertices are written
        ya = __double_as_longlong(fx::to_double_cvt(nw.a, c.R - fx::FRAC));
        yb = __double_as_longlong(fx::to_double_cvt(nw.b, c.R - fx::FRAC));
      }
      long long *yrow = (long long *)yplane + (int64_t)j * c.pitch;
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
}

template <bool FIXA, int XF, int NF, int YF, bool INNER>
__device__ void run_half_t(Ctx &c, int pz, int i0, int i1, const void *F, void *Y, long long *sm, uint64_t *bars,
                           int *fail, const CUtensorMap *mapX, const CUtensorMap *mapN, long long &vmax) {
  const Geo &q = c.q;
  auto slot = [&](int i) -> long long * { return sm + i * GT_SLOT; };
  unsigned ph = 0;    // bit s: parity of the next completion on slot s
  unsigned pend = 0;  // bit s: a load into slot s not yet waited for
  int sl_lo = 0, sl_up = 1, sl_ce = 2, sl_nup = 3, sl_nce = 4;
  auto issue = [&](int s, const CUtensorMap *m, int64_t z) {
    pend |= 1u << s;
    if (threadIdx.x == 0) {
      fence_proxy_async();  // earlier generic accesses to the slot before the TMA writes it
      tma_load_plane(slot(s), m, c.x0 - 2, c.y0 - 2, (int)z, &bars[s], GT_SLOT * 8);
    }
  };
  auto wait = [&](int s) {
    if (!mbar_wait(&bars[s], (ph >> s) & 1u, GT_WAIT)) {
      atomicExch(fail, 1);  // the load stays pending
      return;
    }
    ph ^= 1u << s;
    pend &= ~(1u << s);
  };
  // after a failed wait: wait once more (bounded) for every load still in flight so that
  // none lands in shared memory after the CTA has left
  auto drain = [&]() {
    for (int s = 0; s < GT_NSLOT; ++s)
      if (pend & (1u << s)) mbar_wait(&bars[s], (ph >> s) & 1u, GT_WAIT);
  };
  // bring a staged slot to this sweep's representation (format fmt, extra shift d)
  auto convert = [&](int s, int fmt, int d) {
    if (!FIXA || (fmt == FXP && d == 0)) return;
    long long *p = slot(s);
    for (int idx = threadIdx.x; idx < GT_SLOT; idx += GT_THREADS)
      p[idx] = fmt == F64 ? fx::to_fixed(__longlong_as_double(p[idx]), 1023 + c.R) : shr(p[idx], d);
  };
  const char *Fc = (const char *)F;
  char *Yc = (char *)Y;
  const int64_t P = q.plane;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int xa = c.x0 - 2 + 2 * lane;
  // right-hand sides of this warp's rows: phase 1 rows 2+4w, 4+4w; phase 2 rows 3+4w, 5+4w
  auto load_f = [&](int64_t z, LP (&f1)[2], LP (&f2)[2]) {
    const bool zin = z >= 1 && z <= q.nz - 1;
    const void *fp = zin ? Fc + z * P * 8 : nullptr;
    for (int k = 0; k < 2; ++k) {
      f1[k] = ld_rhs<INNER>(c, fp, c.y0 - 2 + 2 + 4 * warp + 2 * k, xa);
      f2[k] = ld_rhs<INNER>(c, fp, c.y0 - 2 + 3 + 4 * warp + 2 * k, xa);
    }
  };
  {
    const int64_t z = pz + 2 * (int64_t)i0;
    issue(sl_lo, mapN, z - 1);
    issue(sl_up, mapN, z + 1);
    issue(sl_ce, mapX, z);
    if (i0 + 1 < i1) {
      issue(sl_nce, mapX, z + 2);
      issue(sl_nup, mapN, z + 3);
    }
    wait(sl_lo);
    __syncthreads();
    if (*fail) {
      drain();
      return;
    }
    convert(sl_lo, NF, c.dn);
  }
  LP f1[2], f2[2];
  load_f(pz + 2 * (int64_t)i0, f1, f2);
  for (int i = i0; i < i1; ++i) {
    const int64_t z = pz + 2 * (int64_t)i;
    const bool zin = z >= 1 && z <= q.nz - 1;
    wait(sl_ce);
    wait(sl_up);
    __syncthreads();
    if (*fail) {  // a TMA wait ran out
      drain();
      return;
    }
    convert(sl_up, NF, c.dn);
    convert(sl_ce, XF, c.dx);
    __syncthreads();
    const LP g1[2] = {f1[0], f1[1]}, g2[2] = {f2[0], f2[1]};
    if (i + 1 < i1) load_f(z + 2, f1, f2);
    void *yp = Yc + z * P * 8;
    if (zin) {
      phase_t<FIXA, YF, INNER, 1>(c, slot(sl_ce), slot(sl_lo), slot(sl_up), yp, g1, vmax);
      __syncthreads();
      phase_t<FIXA, YF, INNER, 2>(c, slot(sl_ce), slot(sl_lo), slot(sl_up), yp, g2, vmax);
    } else if (c.write_bnd) {
      // Dirichlet plane (fixed-point output): carry the core through
      const long long *cs = slot(sl_ce);
      for (int idx = threadIdx.x; idx < GT_TX * GT_TY; idx += GT_THREADS) {
        const int x = c.x0 + idx % GT_TX, j = c.y0 + idx / GT_TX;
        if (x > c.nx || j > c.ny) continue;
        const long long v = cs[(j - c.y0 + 2) * GT_W + (x - c.x0 + 2)];
        ((long long *)yp)[(int64_t)j * c.pitch + x] = v;
        const long long m = FIXA ? (v < 0 ? -v : v) : (long long)fx::abs_bits(__longlong_as_double(v));
        vmax = max(vmax, m);
      }
    }
    __syncthreads();  // every access to the freed slots is done
    // rotate: N(z+1) becomes the lower neighbour, the in-flight planes the current ones
    const int t_lo = sl_lo, t_ce = sl_ce;
    sl_lo = sl_up;
    sl_up = sl_nup;
    sl_ce = sl_nce;
    sl_nup = t_lo;
    sl_nce = t_ce;
    if (i + 2 < i1) {
      issue(sl_nce, mapX, z + 4);
      issue(sl_nup, mapN, z + 5);
    }
  }
}

template <int XF, int NF, int YF>
__global__ void __launch_bounds__(GT_THREADS, 2)
    k_gs_half_t(Geo q, int pz, const void *X, const void *N, void *Y, const double *f, const long long *GF,
                SweepBounds *bnd, int sweep, int sweeps, double g, int cz, bool write_bnd,
                const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapN) {
  extern __shared__ unsigned char gt_raw[];
  __shared__ __align__(8) uint64_t bars[GT_NSLOT];
  __shared__ long long red[GT_THREADS / 32];
  __shared__ int fail;
  long long *sm = (long long *)(((uintptr_t)gt_raw + 127) & ~(uintptr_t)127);
  Ctx c;
  c.q = q;
  c.x0 = (int)blockIdx.x * GT_TX;
  c.y0 = (int)blockIdx.y * GT_TY;
  c.g = g;
  c.nx = (int)q.nx;
  c.ny = (int)q.ny;
  c.pitch = (int)q.pitch;
  c.write_bnd = write_bnd;
  const Plan plan = make_plan(bnd, g, sweeps);
  const int rd = sweep % 4, wr = (sweep + 1) % 4, cl = (sweep + 2) % 4;
  c.R = sweep_R(bnd, rd, g);
  const int Rx = sweep > 0 ? sweep_R(bnd, (sweep + 3) % 4, g) : c.R;
  c.dx = XF == FXP ? c.R - Rx : 0;
  c.dn = NF == FXP ? (pz == 0 ? c.dx : 0) : 0;
  // R >= Rf (the sweep's bound includes 4 (3/8) h^2 max|f|): GF needs a right shift,
  // clamped at 63 (which leaves 0 or -1, below one unit of the last place)
  c.df = min(c.R - plan.Rf, 63);
  if (pz == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) bnd->umax[cl] = 0ull;
  if (threadIdx.x == 0) {
    for (int i = 0; i < GT_NSLOT; ++i) mbar_init(&bars[i], 1);
    fail = 0;
    fence_mbar_init();
    fence_proxy_async();
  }
  __syncthreads();
  const int ncentre = q.nz >= pz ? (int)((q.nz - pz) / 2 + 1) : 0;
  const int i0 = (int)blockIdx.z * cz;
  const int i1 = i0 + cz < ncentre ? i0 + cz : ncentre;
  // every computed vertex (staged columns 1..62, rows 1..32) interior
  const bool inner = c.x0 - 1 >= 1 && c.x0 + 60 <= c.nx - 1 && c.y0 - 1 >= 1 && c.y0 + 30 <= c.ny - 1;
  long long vmax = 0;
  if (i0 < i1) {
    if (plan.fix) {
      if (inner)
        run_half_t<true, XF, NF, YF, true>(c, pz, i0, i1, GF, Y, sm, bars, &fail, &mapX, &mapN, vmax);
      else
        run_half_t<true, XF, NF, YF, false>(c, pz, i0, i1, GF, Y, sm, bars, &fail, &mapX, &mapN, vmax);
    } else {
      run_half_t<false, F64, F64, F64, false>(c, pz, i0, i1, f, Y, sm, bars, &fail, &mapX, &mapN, vmax);
    }
  }
  __syncthreads();
  if (fail && threadIdx.x == 0) atomicExch(&g_gs_tma_error, 1u);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long w = __shfl_xor_sync(0xffffffffu, vmax, o);
    vmax = w > vmax ? w : vmax;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = vmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long m = 0;
    for (int w = 0; w < GT_THREADS / 32; ++w) m = red[w] > m ? red[w] : m;
    const unsigned long long mb =
        plan.fix ? fx::abs_bits(fx::to_double(m, c.R - fx::FRAC) * (1.0 + 0x1p-50)) : (unsigned long long)m;
    atomicMax(&bnd->umax[wr], mb);
  }
}

// 3/8 h^2 f in fixed point (scale Rf of the plan) on interior vertices, 0 elsewhere.
__global__ void __launch_bounds__(256) k_prep_gf(Geo q, int dim, const double *__restrict__ f,
                                                 long long *__restrict__ GF, const SweepBounds *bnd, double g,
                                                 int sweeps) {
  const Plan plan = make_plan(bnd, g, sweeps);
  if (!plan.fix) return;
  const int rb = 1023 + plan.Rf;
  const int64_t nrows = (q.nz + 1) * (q.ny + 1);
  for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int64_t k = row / (q.ny + 1), j = row % (q.ny + 1);
    const bool row_inner = j > 0 && j < q.ny && (dim == 2 || (k > 0 && k < q.nz));
    const int64_t base = k * q.plane + j * q.pitch;
    for (int64_t i = threadIdx.x; i <= q.nx; i += blockDim.x)
      GF[base + i] = (row_inner && i > 0 && i < q.nx) ? fx::to_fixed(g * f[base + i], rb) : 0ll;
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
    atomicMax(&bnd->m0, mu);
    atomicMax(&bnd->fmax, mf);
  }
}

}  // namespace

size_t gs_fx_bounds_bytes() { return sizeof(SweepBounds); }

cudaError_t launch_gs_prepass(const Geo &q, int dim, const double *u, const double *f, long long *GF, void *bounds,
                              int sweeps, cudaStream_t s) {
  SweepBounds *bnd = (SweepBounds *)bounds;
  cudaError_t e = cudaMemsetAsync(bnd, 0, sizeof(SweepBounds), s);
  if (e != cudaSuccess) return e;
  const unsigned nb = (unsigned)(8 * device_sm_count());
  k_absmax_uf<<<nb, 256, 0, s>>>(q, dim, u, f, bnd);
  k_prep_gf<<<nb, 256, 0, s>>>(q, dim, f, GF, bnd, 0.375 * q.h * q.h, sweeps);
  return cudaGetLastError();
}

template <int XF, int NF, int YF>
static cudaError_t launch_half(const Geo &q, int pz, const void *X, const void *N, void *Y, const double *f,
                               const long long *GF, SweepBounds *bnd, int sweep, int sweeps, double g,
                               bool write_bnd, cudaStream_t s) {
  static PerDeviceOnce attr;
  {
    cudaError_t e = set_smem_limit_once(attr, k_gs_half_sweep<XF, NF, YF>, GS_SMEM);
    if (e != cudaSuccess) return e;
  }
  const unsigned tx = (unsigned)((q.nx + 1 + GS_TX - 1) / GS_TX);
  const unsigned ty = (unsigned)((q.ny + 1 + GS_TY - 1) / GS_TY);
  const int64_t ncentre = (q.nz - pz) / 2 + 1;
  const int cz = z_chunk((int64_t)tx * ty, ncentre, GS_CZ, 2, 4);
  const unsigned tz = (unsigned)((ncentre + cz - 1) / cz);
  if (ty > 65535 || tz > 65535) return cudaErrorInvalidConfiguration;
  k_gs_half_sweep<XF, NF, YF><<<dim3(tx, ty, tz), GS_THREADS, GS_SMEM, s>>>(q, pz, X, N, Y, f, GF, bnd, sweep,
                                                                            sweeps, g, cz, write_bnd);
  return cudaGetLastError();
}

// TMA-staged half sweep; false (nothing launched) when the arrays do not allow it.
template <int XF, int NF, int YF>
static bool launch_half_t(const Geo &q, int pz, const void *X, const void *N, void *Y, const double *f,
                          const long long *GF, SweepBounds *bnd, int sweep, int sweeps, double g, bool write_bnd,
                          cudaStream_t s, cudaError_t *err) {
  if (((uintptr_t)Y | (uintptr_t)f | (uintptr_t)GF) % 16) return false;
  CUtensorMap mx, mn;
  if (!tma_plane_map(q, X, GT_W, GT_H, &mx) || !tma_plane_map(q, N, GT_W, GT_H, &mn)) return false;
  static PerDeviceOnce attr;
  *err = set_smem_limit_once(attr, k_gs_half_t<XF, NF, YF>, GT_SMEM);
  if (*err != cudaSuccess) return true;
  const unsigned tx = (unsigned)((q.nx + 1 + GT_TX - 1) / GT_TX);
  const unsigned ty = (unsigned)((q.ny + 1 + GT_TY - 1) / GT_TY);
  const int64_t ncentre = (q.nz - pz) / 2 + 1;
  const int cz = tuned_chunk(tuning_lookup(STENCIL_CALL_SMOOTH_COLOURED, q),
                             z_chunk((int64_t)tx * ty, ncentre, GS_CZ, 2, 2), 2, GS_CZ);
  const unsigned tz = (unsigned)((ncentre + cz - 1) / cz);
  if (ty > 65535 || tz > 65535) {
    *err = cudaErrorInvalidConfiguration;
    return true;
  }
  k_gs_half_t<XF, NF, YF><<<dim3(tx, ty, tz), GT_THREADS, GT_SMEM, s>>>(q, pz, X, N, Y, f, GF, bnd, sweep, sweeps,
                                                                      g, cz, write_bnd, mx, mn);
  *err = cudaGetLastError();
  return true;
}

// The TMA-staged kernel where it applies, k_gs_half_sweep otherwise.
template <int XF, int NF, int YF>
static cudaError_t launch_half_any(const Geo &q, int pz, const void *X, const void *N, void *Y, const double *f,
                                   const long long *GF, SweepBounds *bnd, int sweep, int sweeps, double g,
                                   bool write_bnd, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (launch_half_t<XF, NF, YF>(q, pz, X, N, Y, f, GF, bnd, sweep, sweeps, g, write_bnd, s, &e)) return e;
  return launch_half<XF, NF, YF>(q, pz, X, N, Y, f, GF, bnd, sweep, sweeps, g, write_bnd, s);
}

// work: 3 arrays of u's span (8 bytes per element): two ping-pong buffers and GF.
cudaError_t launch_gs_sweeps_fx3(const Geo &q, double *u, const double *f, int sweeps, double *work,
                                 void *bounds, cudaStream_t s) {
  if (q.plane >= ((int64_t)1 << 31) - GS_SW * GS_SH) return cudaErrorInvalidValue;
  const int64_t span = span_elems(q);
  void *A = work, *B = work + span;
  long long *GF = (long long *)(work + 2 * span);
  SweepBounds *bnd = (SweepBounds *)bounds;
  cudaError_t e = launch_gs_prepass(q, 3, u, f, GF, bounds, sweeps, s);
  if (e != cudaSuccess) return e;
  const double g = 0.375 * q.h * q.h;
  if (sweeps == 1) {
    // u -> A in FP64 (boundary carried), then back into u
    e = launch_half<F64, F64, F64>(q, 0, u, u, A, f, GF, bnd, 0, 1, g, true, s);
    if (!e) e = launch_half<F64, F64, F64>(q, 1, u, A, A, f, GF, bnd, 0, 1, g, true, s);
    if (!e) e = cudaMemcpyAsync(u, A, (size_t)span * sizeof(double), cudaMemcpyDeviceToDevice, s);
    return e;
  }
  const void *X = u;
  for (int it = 0; it < sweeps && !e; ++it) {
    const bool first = it == 0, last = it == sweeps - 1;
    void *Y = last ? (void *)u : (it % 2 == 0 ? A : B);
    if (first) {
      e = launch_half_any<F64, F64, FXP>(q, 0, X, X, Y, f, GF, bnd, it, sweeps, g, true, s);
      if (!e) e = launch_half_any<F64, FXP, FXP>(q, 1, X, Y, Y, f, GF, bnd, it, sweeps, g, true, s);
    } else if (!last) {
      e = launch_half_any<FXP, FXP, FXP>(q, 0, X, X, Y, f, GF, bnd, it, sweeps, g, true, s);
      if (!e) e = launch_half_any<FXP, FXP, FXP>(q, 1, X, Y, Y, f, GF, bnd, it, sweeps, g, true, s);
    } else {
      // the caller's u: its Dirichlet values were never overwritten, leave them
      e = launch_half_any<FXP, FXP, F64>(q, 0, X, X, Y, f, GF, bnd, it, sweeps, g, false, s);
      if (!e) e = launch_half_any<FXP, F64, F64>(q, 1, X, Y, Y, f, GF, bnd, it, sweeps, g, false, s);
    }
    X = Y;
  }
  return e ? e : cudaGetLastError();
}

}  // namespace stencil

namespace stencil {

// The TMA wait flag of this file's kernels (1 once a bounded wait ran out); cleared on
// request.  Synchronous.
cudaError_t tma_wait_flag_gs3(unsigned *value, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(value, g_gs_tma_error, sizeof(unsigned));
  if (e == cudaSuccess && clear && *value) {
    const unsigned zero = 0u;
    e = cudaMemcpyToSymbol(g_gs_tma_error, &zero, sizeof(unsigned));
  }
  return e;
}

}  // namespace stencil
