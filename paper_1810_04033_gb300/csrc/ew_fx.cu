// Element-wise (cell-wise) 3D Q1 apply on the integer pipes: every cell computes
// K_e u_e and adds it into its 8 vertices, with the 2^3 cell colours resolving the
// races of the scatter (Section 2: cell-wise weighted sums; Section 3: colouring).
//
// Per cell, 12 K_e/h (the Q1 element matrix scaled to integers: 4 on the diagonal, 0
// for vertices differing in one coordinate, -1 otherwise) gives, for local vertex w,
//   12 (K u_e)_w = 5 u_w + F_w - T,   F_w = sum of the 3 face-adjacent vertices of w,
//   T = sum of all 8 vertex values of the cell,
// evaluated exactly in int64 fixed point (fixed.cuh), so the accumulated vertex sums
// do not depend on the order of the additions.  In fixed point the cell adds -G_w to
// vertex w, 12 (K u_e)_w = 4 u_w - G_w with G_w = T - u_w - F_w (the four vertices that
// share no edge with w), and the 4 u_w parts of a vertex's eight cells are added once,
// as 32 u_w: the same integer sum with fewer operations per cell.  y = sum / (12 h^2)
// on interior vertices, 0 on the boundary.
//
// The scatter runs in registers, one warp per column of cells (layout below): the z
// colours are the cell layers processed in order, the y colours the cell rows processed
// one after the other, and the x colours meet in registers and through shuffles, each
// vertex column being owned by one lane.  After layer k, vertex plane k has received all 8
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

// ------------------------------------------------------------ plane-staged form
// A warp owns a window of 64 vertex columns, two per lane (xa even, xb = xa + 1; lanes
// 1..30 own the 60 output columns), E3_R vertex rows y and a chunk of planes, and
// streams the cell layers k in z order.  Rows j0-1 .. j0+E3_R of each plane are copied
// into the warp's own shared-memory slots with cp.async (zero-filled outside the grid)
// two planes ahead of use, and converted to fixed point in place; the sums of plane k
// (contributions of layers k-1 and k) and the partial sums of plane k+1 (layer k) stay
// in registers.  A lane has two cells per cell row: A (from xa to xb) and B (from xb to
// the next lane's xa, read from the staged plane).  B's shares for the next lane's xa
// column are summed per vertex row and handed over by one shuffle per row once the
// layer is done (the x colours meet there); the y colours are the cell rows processed
// one after the other, the z colours the layers in order; after layer k, plane k has all
// 8 shares and is written.  The fixed-point reference is per warp and only grows (as in
// the 2D kernels); a warp that meets a value outside the fixed-point range switches to
// FP64 at a layer start.
constexpr int E3_R = 4;                         // output vertex rows per warp
constexpr int E3_ROWS = E3_R + 2;               // staged rows per plane
constexpr int E3_W = 64;                        // staged columns
constexpr int E3_BUF = E3_ROWS * E3_W;          // elements per staged plane
constexpr int E3_CZ = 32;                       // output planes per warp (at most)
constexpr int E3_THREADS = 128;
constexpr int E3_OUT = 60;                      // output columns per warp
constexpr size_t E3_SMEM = (size_t)(E3_THREADS / 32) * 3 * E3_BUF * sizeof(long long);
constexpr int E3_RMIN = -900, E3_RMAX = 1000;
// Every lane evaluates both of its cells, also where a cell lies outside the grid (its
// shares then land only on boundary vertices, whose output is 0, or on columns that
// are not written): no divergent branch per cell.
constexpr bool E3_ALLCELLS = true;
constexpr bool E3_SPLIT = false;  // output conversion split between the pipes (measured slower here)

struct P2 {
  long long a, b;  // columns xa, xb
};

struct Ew3Lane {
  int64_t xa;
  bool oka, okb, ina, inb, cellA, cellB, out_lane;
  int lane;
  long long *buf;     // the warp's 3 plane slots
  P2 acc[E3_R];       // plane k rows j0 .. j0+R-1
  long long accR[E3_R];  // shares of plane k for the next lane's xa column
  int R;
};

__device__ __forceinline__ unsigned bexp(double v) { return (unsigned)(fx::dbits(v) >> 52) & 0x7ffu; }

__device__ __forceinline__ long long shr_pos(long long v, int d) { return d >= 63 ? (v >> 63) : (v >> d); }

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Slot of plane z (planes z0-1, z0, z0+1, ... rotate through 3 slots).
__device__ __forceinline__ long long *e3_slot(const Ew3Lane &L, int64_t z, int64_t z0) {
  return L.buf + ((z - z0 + 1) % 3) * E3_BUF;
}

// Start the copy of plane z's staged rows (this lane's two columns) into its slot;
// zeros outside the grid.  One commit group per plane (empty when z is not needed).
template <bool V16>
__device__ __forceinline__ void e3_issue(const EwArgs &a, const Ew3Lane &L, int64_t z, int64_t z0, int64_t j0,
                                         bool need) {
  const Geo &q = a.q;
  if (need) {
    long long *slot = e3_slot(L, z, z0) + 2 * L.lane;
    const long long *base = (const long long *)a.u;
#pragma unroll
    for (int c = 0; c < E3_ROWS; ++c) {
      const int64_t j = j0 - 1 + c;
      const bool row = z >= 0 && z <= q.nz && j >= 0 && j <= q.ny;
      const long long *src = row && L.oka ? base + z * q.plane + j * q.pitch + L.xa : base;
      const uint32_t dst = smem_addr(slot + c * E3_W);
      if (V16) {
        const int bytes = row && L.oka ? (L.okb ? 16 : 8) : 0;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
      } else {
        const int ba = row && L.oka ? 8 : 0, bb = row && L.okb ? 8 : 0;
        const long long *srcb = row && L.okb ? base + z * q.plane + j * q.pitch + L.xa + 1 : base;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(ba) : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst + 8), "l"(srcb), "r"(bb) : "memory");
      }
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// 12 K_e u_e of one cell (bottom face b0..b3, top face t0..t3; index bit 0 = x, bit 1 =
// y): cb_w for the bottom vertices, ct_w for the top ones.
template <bool FIX>
__device__ __forceinline__ void cell12(long long b0, long long b1, long long b2, long long b3, long long t0,
                                       long long t1, long long t2, long long t3, long long (&cb)[4],
                                       long long (&ct)[4]) {
  const long long Sb = add<FIX>(add<FIX>(b0, b1), add<FIX>(b2, b3));
  const long long St = add<FIX>(add<FIX>(t0, t1), add<FIX>(t2, t3));
  cb[0] = add<FIX>(sub<FIX>(times4<FIX>(b0), b3), sub<FIX>(t0, St));
  cb[1] = add<FIX>(sub<FIX>(times4<FIX>(b1), b2), sub<FIX>(t1, St));
  cb[2] = add<FIX>(sub<FIX>(times4<FIX>(b2), b1), sub<FIX>(t2, St));
  cb[3] = add<FIX>(sub<FIX>(times4<FIX>(b3), b0), sub<FIX>(t3, St));
  ct[0] = add<FIX>(sub<FIX>(times4<FIX>(t0), t3), sub<FIX>(b0, Sb));
  ct[1] = add<FIX>(sub<FIX>(times4<FIX>(t1), t2), sub<FIX>(b1, Sb));
  ct[2] = add<FIX>(sub<FIX>(times4<FIX>(t2), t1), sub<FIX>(b2, Sb));
  ct[3] = add<FIX>(sub<FIX>(times4<FIX>(t3), t0), sub<FIX>(b3, Sb));
}

// Fixed-point form of the same cell: 12 (K u_e)_w = 4 u_w - G_w, G_w = the sum of the
// four cell vertices that share no edge with w (the three face diagonals and the body
// diagonal); gb / gt receive G_w of the bottom / top vertices.  The 4 u_w parts of a
// vertex's eight cells are added once, as 32 u_w, when its plane is complete.
__device__ __forceinline__ void cell_g(long long b0, long long b1, long long b2, long long b3, long long t0,
                                       long long t1, long long t2, long long t3, long long (&gb)[4],
                                       long long (&gt)[4]) {
  const long long Sb = (b0 + b1) + (b2 + b3), St = (t0 + t1) + (t2 + t3);
  gb[0] = b3 + St - t0;
  gb[1] = b2 + St - t1;
  gb[2] = b1 + St - t2;
  gb[3] = b0 + St - t3;
  gt[0] = t3 + Sb - b0;
  gt[1] = t2 + Sb - b1;
  gt[2] = t1 + Sb - b2;
  gt[3] = t0 + Sb - b3;
}

// This lane's staged pair of row c and the next lane's xa value of that row.
struct Row3 {
  long long a, b, r;
};

__device__ __forceinline__ Row3 e3_row(const long long *plane, int c, int lane) {
  const longlong2 v = *(const longlong2 *)(plane + c * E3_W + 2 * lane);
  const int rc = lane < 31 ? 2 * lane + 2 : 2 * lane;  // lane 31 has no cell B
  return Row3{v.x, v.y, plane[c * E3_W + rc]};
}

// Layers k0 .. z1-1 of the warp's column; returns the first layer not done (the warp
// switched to FP64) or z1.  resume: plane k0+1 is already waited for and k0+2 issued.
template <bool FIX, bool V16>
__device__ __forceinline__ int64_t ew3_layers(const EwArgs &a, Ew3Lane &L, int64_t j0, int64_t z0, int64_t z1,
                                              int64_t k0, bool resume) {
  const Geo &q = a.q;
  const long long zero = FIX ? 0ll : __double_as_longlong(0.0);
  long long *own = nullptr;
  for (int64_t k = k0; k < z1; ++k) {
    if (!(resume && k == k0)) {
      e3_issue<V16>(a, L, k + 2, z0, j0, k + 2 <= z1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
      __syncwarp();
    }
    long long *bot = e3_slot(L, k, z0), *top = e3_slot(L, k + 1, z0);
    own = top + 2 * L.lane;
    if (FIX) {
      unsigned em = 0;
#pragma unroll
      for (int c = 0; c < E3_ROWS; ++c) {
        const longlong2 v = *(const longlong2 *)(own + c * E3_W);
        em = max(em, max(bexp(__longlong_as_double(v.x)), bexp(__longlong_as_double(v.y))));
      }
      em = __reduce_max_sync(0xffffffffu, em);
      if (em != 0) {
        const int Rp = (int)em - 1022 + 1;
        long long *ob = bot + 2 * L.lane;
        if (em == 2047 || Rp > E3_RMAX || (Rp < E3_RMIN && L.R == E3_RMIN)) {
          if (k >= 1 && k <= q.nz) {
            // the 4 u_v parts of layer k-1's cells: 2 cells (A) at xa, 4 at xb, 2 (B) at
            // the next lane's xa, for each vertex row
#pragma unroll
            for (int r = 0; r < E3_R; ++r) {
              const long long *row = ob + (r + 1) * E3_W;
              L.acc[r].a += 8 * row[0];
              L.acc[r].b += 16 * row[1];
              L.accR[r] += 8 * row[2];
            }
          }
          auto cv = [&](long long v) { return __double_as_longlong(fx::to_double(v, L.R - fx::FRAC)); };
#pragma unroll
          for (int c = 0; c < E3_ROWS; ++c) {
            ob[c * E3_W] = cv(ob[c * E3_W]);
            ob[c * E3_W + 1] = cv(ob[c * E3_W + 1]);
          }
#pragma unroll
          for (int r = 0; r < E3_R; ++r) {
            L.acc[r] = P2{cv(L.acc[r].a), cv(L.acc[r].b)};
            L.accR[r] = cv(L.accR[r]);
          }
          __syncwarp();
          return k;  // redo this layer in FP64
        }
        if (Rp > L.R) {
          const int d = Rp - L.R;
#pragma unroll
          for (int c = 0; c < E3_ROWS; ++c) {
            ob[c * E3_W] = shr_pos(ob[c * E3_W], d);
            ob[c * E3_W + 1] = shr_pos(ob[c * E3_W + 1], d);
          }
#pragma unroll
          for (int r = 0; r < E3_R; ++r) {
            L.acc[r] = P2{shr_pos(L.acc[r].a, d), shr_pos(L.acc[r].b, d)};
            L.accR[r] = shr_pos(L.accR[r], d);
          }
          L.R = Rp;
        }
      }
#pragma unroll
      for (int c = 0; c < E3_ROWS; ++c) {
        longlong2 *p = (longlong2 *)(own + c * E3_W);
        const longlong2 v = *p;
        *p = make_longlong2(fx::to_fixed(__longlong_as_double(v.x), 1023 + L.R),
                            fx::to_fixed(__longlong_as_double(v.y), 1023 + L.R));
      }
      __syncwarp();
    }
    P2 part[E3_R];
    long long partR[E3_R];
#pragma unroll
    for (int r = 0; r < E3_R; ++r) {
      part[r] = P2{zero, zero};
      partR[r] = zero;
    }
    if (k >= 0 && k < q.nz) {
      Row3 b0 = e3_row(bot, 0, L.lane), t0 = e3_row(top, 0, L.lane);
#pragma unroll
      for (int c = 0; c <= E3_R; ++c) {
        const Row3 b1 = e3_row(bot, c + 1, L.lane), t1 = e3_row(top, c + 1, L.lane);
        const int64_t cj = j0 - 1 + c;
        if (cj >= 0 && cj < q.ny) {  // warp-uniform
          long long cb[4], ct[4];
          if (FIX) {
            long long gb[4], gt[4];
            cell_g(b0.a, b0.b, b1.a, b1.b, t0.a, t0.b, t1.a, t1.b, gb, gt);  // cell A
            if (c >= 1) {
              L.acc[c - 1].a -= gb[0];
              L.acc[c - 1].b -= gb[1];
              part[c - 1].a -= gt[0];
              part[c - 1].b -= gt[1];
            }
            if (c < E3_R) {
              L.acc[c].a -= gb[2];
              L.acc[c].b -= gb[3];
              part[c].a -= gt[2];
              part[c].b -= gt[3];
            }
            cell_g(b0.b, b0.r, b1.b, b1.r, t0.b, t0.r, t1.b, t1.r, gb, gt);  // cell B
            if (c >= 1) {
              L.acc[c - 1].b -= gb[0];
              L.accR[c - 1] -= gb[1];
              part[c - 1].b -= gt[0];
              partR[c - 1] -= gt[1];
            }
            if (c < E3_R) {
              L.acc[c].b -= gb[2];
              L.accR[c] -= gb[3];
              part[c].b -= gt[2];
              partR[c] -= gt[3];
            }
          } else if (E3_ALLCELLS || L.cellA) {  // vertices xa, xb of rows cj, cj+1
            cell12<FIX>(b0.a, b0.b, b1.a, b1.b, t0.a, t0.b, t1.a, t1.b, cb, ct);
            if (c >= 1) {
              L.acc[c - 1].a = add<FIX>(L.acc[c - 1].a, cb[0]);
              L.acc[c - 1].b = add<FIX>(L.acc[c - 1].b, cb[1]);
              part[c - 1].a = add<FIX>(part[c - 1].a, ct[0]);
              part[c - 1].b = add<FIX>(part[c - 1].b, ct[1]);
            }
            if (c < E3_R) {
              L.acc[c].a = add<FIX>(L.acc[c].a, cb[2]);
              L.acc[c].b = add<FIX>(L.acc[c].b, cb[3]);
              part[c].a = add<FIX>(part[c].a, ct[2]);
              part[c].b = add<FIX>(part[c].b, ct[3]);
            }
          }
          if (!FIX && (E3_ALLCELLS || L.cellB)) {  // vertices xb and the next lane's xa
            cell12<FIX>(b0.b, b0.r, b1.b, b1.r, t0.b, t0.r, t1.b, t1.r, cb, ct);
            if (c >= 1) {
              L.acc[c - 1].b = add<FIX>(L.acc[c - 1].b, cb[0]);
              L.accR[c - 1] = add<FIX>(L.accR[c - 1], cb[1]);
              part[c - 1].b = add<FIX>(part[c - 1].b, ct[0]);
              partR[c - 1] = add<FIX>(partR[c - 1], ct[1]);
            }
            if (c < E3_R) {
              L.acc[c].b = add<FIX>(L.acc[c].b, cb[2]);
              L.accR[c] = add<FIX>(L.accR[c], cb[3]);
              part[c].b = add<FIX>(part[c].b, ct[2]);
              partR[c] = add<FIX>(partR[c], ct[3]);
            }
          }
        }
        b0 = b1;
        t0 = t1;
      }
    }
    // plane k complete: the left lane's B shares land on this lane's xa column
#pragma unroll
    for (int r = 0; r < E3_R; ++r) {
      long long l = __shfl_up_sync(0xffffffffu, L.accR[r], 1);
      if (L.lane == 0) l = zero;
      L.acc[r].a = add<FIX>(L.acc[r].a, l);
    }
    if (k >= z0 && k <= q.nz && L.out_lane) {
      const bool zin = k >= 1 && k < q.nz;
      long long *out = (long long *)a.y + k * q.plane;
      // scale 2^(R-52) / (12 h^2), exact power-of-two scaling of a.scale
      const double sc = FIX ? a.scale * fx::pow2d(L.R - fx::FRAC) : a.scale;
#pragma unroll
      for (int r = 0; r < E3_R; ++r) {
        const int64_t j = j0 + r;
        if (j > q.ny) break;
        const bool jin = zin && j >= 1 && j < q.ny;
        // the odd column converts with integer instructions (E3_SPLIT), moving a quarter
        // of the conversions' FP64-pipe work to the integer pipes; the same bits
        long long sa = L.acc[r].a, sbv = L.acc[r].b;
        if (FIX) {  // the 4 u_v parts of the eight cells
          const longlong2 uk = *(const longlong2 *)(bot + (r + 1) * E3_W + 2 * L.lane);
          sa += 32 * uk.x;
          sbv += 32 * uk.y;
        }
        const double va = FIX ? __ll2double_rn(sa) : __longlong_as_double(sa);
        const double vb = !FIX ? __longlong_as_double(sbv)
                          : E3_SPLIT ? fx::to_double(sbv, L.R - fx::FRAC) : __ll2double_rn(sbv);
        const double sb = FIX && E3_SPLIT ? a.scale : sc;
        const long long ya = __double_as_longlong(jin && L.ina ? va * sc : 0.0);
        const long long yb = __double_as_longlong(jin && L.inb ? vb * sb : 0.0);
        long long *row = out + j * q.pitch;
        if (V16 && L.oka && L.okb) {
          *(longlong2 *)(row + L.xa) = make_longlong2(ya, yb);
        } else {
          if (L.oka) row[L.xa] = ya;
          if (L.okb) row[L.xa + 1] = yb;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < E3_R; ++r) {
      L.acc[r] = part[r];
      L.accR[r] = partR[r];
    }
    __syncwarp();  // every lane is done with plane k's slot before it is refilled
  }
  return z1;
}

template <bool V16>
__global__ void __launch_bounds__(E3_THREADS) k_apply_elementwise_s3(EwArgs a) {
  extern __shared__ long long e3_smem[];
  const Geo &q = a.q;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * (E3_THREADS / 32) + wib;
  const int64_t nseg = (q.nx + E3_OUT) / E3_OUT, njc = (q.ny + E3_R) / E3_R;
  const int64_t seg = gw % nseg, rest = gw / nseg;
  const int64_t jc = rest % njc, zc = rest / njc;
  const int64_t z0 = zc * a.cz;
  if (z0 > q.nz) return;
  const int64_t z1 = z0 + a.cz < q.nz + 1 ? z0 + a.cz : q.nz + 1;
  const int64_t j0 = jc * E3_R;
  Ew3Lane L;
  L.lane = lane;
  L.buf = e3_smem + (size_t)wib * 3 * E3_BUF;
  L.xa = seg * E3_OUT - 2 + 2 * lane;
  L.oka = L.xa >= 0 && L.xa <= q.nx;
  L.okb = L.xa + 1 >= 0 && L.xa + 1 <= q.nx;
  L.ina = L.xa >= 1 && L.xa < q.nx;
  L.inb = L.xa + 1 >= 1 && L.xa + 1 < q.nx;
  L.cellA = L.xa >= 0 && L.xa < q.nx;
  L.cellB = lane <= 30 && L.xa + 1 >= 0 && L.xa + 1 < q.nx;
  L.out_lane = lane >= 1 && lane <= 30;
  L.R = E3_RMIN;
  // plane z0-1 (the first layer's bottom face) and no contributions yet; plane z0 in
  // flight behind it
  e3_issue<V16>(a, L, z0 - 1, z0, j0, true);
  e3_issue<V16>(a, L, z0, z0, j0, true);
  asm volatile("cp.async.wait_group 1;" ::: "memory");
  __syncwarp();
  bool fix = true;
  {
    long long *own = e3_slot(L, z0 - 1, z0) + 2 * lane;
    unsigned em = 0;
#pragma unroll
    for (int c = 0; c < E3_ROWS; ++c) {
      const longlong2 v = *(const longlong2 *)(own + c * E3_W);
      em = max(em, max(bexp(__longlong_as_double(v.x)), bexp(__longlong_as_double(v.y))));
    }
    em = __reduce_max_sync(0xffffffffu, em);
    if (em != 0) {
      const int Rp = (int)em - 1022 + 1;
      if (em == 2047 || Rp > E3_RMAX || Rp < E3_RMIN)
        fix = false;
      else
        L.R = Rp;
    }
    if (fix) {
#pragma unroll
      for (int c = 0; c < E3_ROWS; ++c) {
        longlong2 *p = (longlong2 *)(own + c * E3_W);
        const longlong2 v = *p;
        *p = make_longlong2(fx::to_fixed(__longlong_as_double(v.x), 1023 + L.R),
                            fx::to_fixed(__longlong_as_double(v.y), 1023 + L.R));
      }
    }
    __syncwarp();
    const long long zero = fix ? 0ll : __double_as_longlong(0.0);
#pragma unroll
    for (int r = 0; r < E3_R; ++r) {
      L.acc[r] = P2{zero, zero};
      L.accR[r] = zero;
    }
  }
  int64_t k = z0 - 1;
  bool resume = false;
  if (fix) {
    k = ew3_layers<true, V16>(a, L, j0, z0, z1, k, false);
    resume = true;  // a switch happens after plane k+1 was waited for
  }
  if (k < z1) ew3_layers<false, V16>(a, L, j0, z0, z1, k, resume);
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

}  // namespace

cudaError_t launch_apply_elementwise_fx3(const Geo &q, const double *u, double *y, cudaStream_t s) {
  const int64_t nseg = (q.nx + E3_OUT) / E3_OUT, njc = (q.ny + E3_R) / E3_R;
  const int cz = tuned_chunk(tuning_lookup(STENCIL_CALL_APPLY_ELEMENTWISE, q), z_chunk(nseg * njc, q.nz + 1, E3_CZ, 4, 64),
                            4, E3_CZ);
  const int64_t nzc = (q.nz + cz) / cz;
  const int64_t warps = nseg * njc * nzc;
  const int64_t blocks = (warps + E3_THREADS / 32 - 1) / (E3_THREADS / 32);
  if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
  EwArgs a;
  a.q = q;
  a.u = u;
  a.y = y;
  a.scale = 1.0 / (12.0 * q.h * q.h);
  a.cz = cz;
  // 16-byte pairs: even pitch (so every plane and row start is even too) and 16-byte
  // aligned arrays
  const bool v16 = q.pitch % 2 == 0 && ((uintptr_t)u % 16) == 0 && ((uintptr_t)y % 16) == 0;
  static PerDeviceOnce attr_t, attr_f;
  {
    cudaError_t e = set_smem_limit_once(attr_t, k_apply_elementwise_s3<true>, E3_SMEM);
    if (!e) e = set_smem_limit_once(attr_f, k_apply_elementwise_s3<false>, E3_SMEM);
    if (e) return e;
  }
  if (v16)
    k_apply_elementwise_s3<true><<<(unsigned)blocks, E3_THREADS, E3_SMEM, s>>>(a);
  else
    k_apply_elementwise_s3<false><<<(unsigned)blocks, E3_THREADS, E3_SMEM, s>>>(a);
  return cudaGetLastError();
}

}  // namespace stencil
