// 2D Q1 (bilinear, 9-point stencil of Fig. 1) operations on the integer pipes:
// assembled apply, element-wise apply with colour passes, damped Jacobi sweep,
// residual with norms, and the coloured Gauss-Seidel half sweeps.
//
//   3 S u = 8 u - N,  N = sum of the 8 neighbours;   6 K_e (element matrix, h-free) has
//   entries 4 (same vertex), -1 (differ in one coordinate), -2 (opposite corner).
// Values are int64 fixed point (fixed.cuh); N is formed from column sums
//   V = u(j-1) + u(j+1),  T = V + u(j),  N(x) = T(x-1) + T(x+1) + V(x).
//
// Each warp owns a segment of 32 consecutive columns and streams down a chunk of rows,
// keeping the rows it needs in registers and reaching x-neighbours by shuffles; no
// shared memory and no block barriers.  The fixed-point reference R is per warp and
// only grows: every newly loaded row is reduced to its largest exponent first, and when
// that exceeds R the rows held so far are shifted to the new scale.  A warp that meets
// a non-finite value or magnitudes outside [2^-900, 2^1000] converts what it holds to
// FP64 and continues in native FP64 arithmetic.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fixed.cuh"
#include "internal.h"

namespace stencil {
namespace {

constexpr int W2_THREADS = 128;
constexpr int W2_ROWS = 64;  // rows per warp
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

__device__ __forceinline__ long long enc(const WarpScale &w, double v) {
  return w.fix ? fx::to_fixed(v, 1023 + w.R) : __double_as_longlong(v);
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

template <int OP>
__global__ void __launch_bounds__(W2_THREADS) k_ops2(Op2Args a) {
  __shared__ double sh[2 * W2_THREADS / 32];
  __shared__ bool last;
  const Geo &q = a.q;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * (W2_THREADS / 32) + wib;
  const int64_t nseg = (q.nx + 30) / 30;  // 30 outputs per segment
  const int64_t seg = gw % nseg, chunk = gw / nseg;
  const int64_t js = chunk * W2_ROWS;
  const int64_t je = js + W2_ROWS < q.ny + 1 ? js + W2_ROWS : q.ny + 1;
  const int64_t x = seg * 30 + lane - 1;  // lanes 1..30 produce outputs
  const bool xok = x >= 0 && x <= q.nx;
  const bool xin = x >= 1 && x < q.nx;
  const bool out_lane = lane >= 1 && lane <= 30 && xok;
  double rr = 0.0, ff = 0.0;
  WarpScale w;
  if (js <= q.ny) {
    auto load = [&](int64_t j) -> double {
      return (xok && j >= 0 && j <= q.ny) ? a.u[j * q.pitch + x] : 0.0;
    };
    if (OP == O2_ELEMENTWISE) {
      // stream cell rows cj = js-1 .. je-1; vertex row cj is complete after cell row cj
      double ra = load(js - 1);
      int d = admit_row(w, __reduce_max_sync(0xffffffffu, biased_exp(ra)), 1);
      if (d < 0) w.fix = false;
      long long ua = enc(w, ra), alo = 0, ahi = 0;
      double rb_next = load(js);
      for (int64_t cj = js - 1; cj < je; ++cj) {
        const double rb = rb_next;
        if (cj + 2 <= je) rb_next = load(cj + 2);
        d = admit_row(w, __reduce_max_sync(0xffffffffu, biased_exp(rb)), 1);
        if (d < 0) {
          ua = to_f64_bits(ua, w.R);
          alo = to_f64_bits(alo, w.R);
          ahi = to_f64_bits(ahi, w.R);
          w.fix = false;
        } else if (d > 0) {
          ua = shr(ua, d);
          alo = shr(alo, d);
          ahi = shr(ahi, d);
        }
        const long long ub = enc(w, rb);
        // the cell with lower-left vertex (x, cj): v0 = (x,cj), v1 = (x+1,cj),
        // v2 = (x,cj+1), v3 = (x+1,cj+1); two colour passes over the x parity
        const long long v1 = __shfl_down_sync(0xffffffffu, ua, 1);
        const long long v3 = __shfl_down_sync(0xffffffffu, ub, 1);
        const bool cell = lane <= 30 && x >= 0 && x < q.nx && cj >= 0 && cj < q.ny;
        for (int px = 0; px < 2; ++px) {
          const bool mine = cell && (int)(x & 1) == px;
          long long c0 = 0, c1 = 0, c2 = 0, c3 = 0;
          if (mine) {
            if (w.fix) {
              c0 = 4 * ua - (v1 + ub) - 2 * v3;
              c1 = 4 * v1 - (ua + v3) - 2 * ub;
              c2 = 4 * ub - (ua + v3) - 2 * v1;
              c3 = 4 * v3 - (v1 + ub) - 2 * ua;
            } else {
              const double A0 = __longlong_as_double(ua), A1 = __longlong_as_double(v1),
                           A2 = __longlong_as_double(ub), A3 = __longlong_as_double(v3);
              c0 = __double_as_longlong(4.0 * A0 - (A1 + A2) - 2.0 * A3);
              c1 = __double_as_longlong(4.0 * A1 - (A0 + A3) - 2.0 * A2);
              c2 = __double_as_longlong(4.0 * A2 - (A0 + A3) - 2.0 * A1);
              c3 = __double_as_longlong(4.0 * A3 - (A1 + A2) - 2.0 * A0);
            }
          }
          // contributions to the right-hand vertices go to the next lane
          const long long c1l = __shfl_up_sync(0xffffffffu, c1, 1);
          const long long c3l = __shfl_up_sync(0xffffffffu, c3, 1);
          if (w.fix) {
            alo += c0 + (lane >= 1 ? c1l : 0);
            ahi += c2 + (lane >= 1 ? c3l : 0);
          } else {
            alo = add<false>(alo, add<false>(c0, lane >= 1 ? c1l : 0));
            ahi = add<false>(ahi, add<false>(c2, lane >= 1 ? c3l : 0));
          }
        }
        if (cj >= js && out_lane) {
          const bool inner = xin && cj >= 1 && cj < q.ny;
          const double s = w.fix ? fx::to_double(alo, w.R - fx::FRAC) : __longlong_as_double(alo);
          a.out[cj * q.pitch + x] = inner ? s * a.c1 : 0.0;
        }
        alo = ahi;
        ahi = 0;
        ua = ub;
      }
    } else {
      // rows j-1, j, j+1 in registers; j+2 in flight
      double rm = load(js - 1), rc = load(js), rp = load(js + 1);
      unsigned em = __reduce_max_sync(0xffffffffu, biased_exp(rm));
      em = max(em, __reduce_max_sync(0xffffffffu, biased_exp(rc)));
      em = max(em, __reduce_max_sync(0xffffffffu, biased_exp(rp)));
      if (admit_row(w, em, 1) < 0) w.fix = false;
      long long um = enc(w, rm), uc = enc(w, rc), up = enc(w, rp);
      double rn = load(js + 2);
      for (int64_t j = js; j < je; ++j) {
        double fv = 0.0;
        const bool inner = xin && j >= 1 && j < q.ny;
        if (OP != O2_APPLY && out_lane && inner) fv = a.f[j * q.pitch + x];
        const long long T = w.fix ? eight_u_minus_n<true>(um, uc, up) : eight_u_minus_n<false>(um, uc, up);
        if (out_lane) {
          const double Td = inner ? (w.fix ? fx::to_double(T, w.R - fx::FRAC) : __longlong_as_double(T)) : 0.0;
          const int64_t gp = j * q.pitch + x;
          if (OP == O2_APPLY) {
            a.out[gp] = inner ? Td * a.c1 : 0.0;
          } else if (OP == O2_JACOBI) {
            a.out[gp] = inner ? fma(a.c2, Td, fma(a.c1, fv, rc)) : rc;
          } else {
            const double r = inner ? fma(a.c1, Td, fv) : 0.0;
            if (a.out) a.out[gp] = r;
            if (inner) {
              rr = fma(r, r, rr);
              ff = fma(fv, fv, ff);
            }
          }
        }
        // advance: admit row j+2
        const double rnn = (j + 3 <= je) ? load(j + 3) : 0.0;
        const int d = admit_row(w, __reduce_max_sync(0xffffffffu, biased_exp(rn)), 1);
        if (d < 0) {
          uc = to_f64_bits(uc, w.R);
          up = to_f64_bits(up, w.R);
          w.fix = false;
        } else if (d > 0) {
          uc = shr(uc, d);
          up = shr(up, d);
        }
        um = uc;
        uc = up;
        up = enc(w, rn);
        rc = rp;
        rp = rn;
        rn = rnn;
      }
    }
  }
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
// Half sweep over the rows of parity pr (0: colours 0, 1; 1: colours 2, 3), out of place
// from X into Y: the centre row comes from X, the rows above and below from N (X for
// the even-row pass, Y for the odd-row pass, which then holds the new even rows).
// Inside a row the even-x colour is updated first; the odd-x colour then reads it
// through shuffles, so a warp produces columns for lanes 2..29 (28 per segment).
// u_new = 3/8 h^2 f + N/8.
__global__ void __launch_bounds__(W2_THREADS) k_gs2_half(Geo q, int pr, const double *__restrict__ X,
                                                         const double *__restrict__ N, double *__restrict__ Y,
                                                         const double *__restrict__ f, double g) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * (W2_THREADS / 32) + wib;
  const int64_t nseg = (q.nx + 28) / 28;
  const int64_t seg = gw % nseg, chunk = gw / nseg;
  const int64_t ncentre = (q.ny - pr) / 2 + 1;
  const int64_t i0 = chunk * (W2_ROWS / 2);
  if (i0 >= ncentre) return;
  const int64_t i1 = i0 + W2_ROWS / 2 < ncentre ? i0 + W2_ROWS / 2 : ncentre;
  const int64_t x = seg * 28 + lane - 2;
  const bool xok = x >= 0 && x <= q.nx;
  const bool xin = x >= 1 && x < q.nx;
  const bool out_lane = lane >= 2 && lane <= 29 && xok;
  WarpScale w;
  auto ld = [&](const double *p, int64_t j) -> double {
    return (xok && j >= 0 && j <= q.ny) ? p[j * q.pitch + x] : 0.0;
  };
  const int64_t jf = pr + 2 * i0;
  double rm = ld(N, jf - 1);
  if (admit_row(w, __reduce_max_sync(0xffffffffu, biased_exp(rm)), 2) < 0) w.fix = false;
  long long um = enc(w, rm);
  for (int64_t i = i0; i < i1; ++i) {
    const int64_t j = pr + 2 * i;
    const bool jin = j >= 1 && j < q.ny;
    const double rc = ld(X, j), rp = ld(N, j + 1);
    const double fv = (jin && xin) ? f[j * q.pitch + x] : 0.0;
    unsigned em = __reduce_max_sync(0xffffffffu, biased_exp(rc));
    em = max(em, __reduce_max_sync(0xffffffffu, biased_exp(rp)));
    em = max(em, __reduce_max_sync(0xffffffffu, biased_exp(g * fv)));
    const int d = admit_row(w, em, 2);  // new values <= max|u| + g max|f|: two spare bits
    if (d < 0) {
      um = to_f64_bits(um, w.R);
      w.fix = false;
    } else if (d > 0) {
      um = shr(um, d);
    }
    long long uc = enc(w, rc);
    const long long up = enc(w, rp);
    double out = rc;
    if (jin) {
      for (int px = 0; px < 2; ++px) {
        const long long V = w.fix ? um + up : add<false>(um, up);
        const long long T = w.fix ? V + uc : add<false>(V, uc);
        const long long Tm = __shfl_up_sync(0xffffffffu, T, 1);
        const long long Tp = __shfl_down_sync(0xffffffffu, T, 1);
        const bool mine = xin && (int)(x & 1) == px;
        if (mine) {
          double un;
          if (w.fix) {
            const long long Nn = Tm + Tp + V;
            un = fma(g, fv, fx::to_double(Nn, w.R - fx::FRAC - 3));
            uc = fx::to_fixed(un, 1023 + w.R);
          } else {
            const double Nn = __longlong_as_double(Tm) + __longlong_as_double(Tp) + __longlong_as_double(V);
            un = fma(Nn, 0.125, g * fv);
            uc = __double_as_longlong(un);
          }
          out = un;
        }
      }
    }
    if (out_lane) Y[j * q.pitch + x] = out;
    um = up;
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

// Coloured GS in 2D: per sweep an even-row pass (X -> Y) and an odd-row pass (new even
// rows from Y); work has u's span.  The result ends in u.
cudaError_t launch_gs_sweeps_fx2(const Geo &q, double *u, const double *f, int sweeps, double *work,
                                 cudaStream_t s) {
  const double g = 0.375 * q.h * q.h;
  const int64_t nseg = (q.nx + 28) / 28;
  const int64_t nchunk = (q.ny + 1 + W2_ROWS - 1) / W2_ROWS + 1;
  const unsigned nb = (unsigned)((nseg * nchunk + W2_THREADS / 32 - 1) / (W2_THREADS / 32));
  double *X = u, *Y = work;
  for (int it = 0; it < sweeps; ++it) {
    k_gs2_half<<<nb, W2_THREADS, 0, s>>>(q, 0, X, X, Y, f, g);
    k_gs2_half<<<nb, W2_THREADS, 0, s>>>(q, 1, X, Y, Y, f, g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double *t = X;
    X = Y;
    Y = t;
  }
  if (X != u) return cudaMemcpyAsync(u, X, (size_t)span_elems(q) * sizeof(double), cudaMemcpyDeviceToDevice, s);
  return cudaSuccess;
}

}  // namespace stencil
