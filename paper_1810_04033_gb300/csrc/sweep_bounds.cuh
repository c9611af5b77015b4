// Per-sweep fixed-point scale shared by the multi-sweep Gauss-Seidel and Jacobi launchers (3D:
// gs_fx.cu and jac3_fx.cu, 2D: ops2d_fx.cu).  Intermediate sweeps keep the iterate in HBM as int64
// fixed point; every value of sweep s is a multiple of 2^(R_s - 52) with |v| < 2^R_s,
// where R_s comes from a bound tracked on the device (no host round trip):
//   B_s = max |u| written by sweep s - 1  +  4 * (3/8) h^2 max |f|,
// the second term covering the growth inside one sweep (each of the 2^d colour
// phases adds at most 3/8 h^2 |f| to a weighted average of its neighbours; in 3D the
// colours are processed as four phases).
#pragma once
#include <stdint.h>

#include "fixed.cuh"

namespace stencil {

// Sweep s reads umax[s % 4] (its bound) and umax[(s + 3) % 4] (the previous sweep's,
// for the scale of its input), accumulates umax[(s + 1) % 4] and clears umax[(s + 2) % 4],
// which no kernel of sweep s reads.
struct SweepBounds {
  unsigned long long umax[4];  // max |u| of the iterate (FP64 bits), ring indexed by sweep
  unsigned long long fmax;     // max |f| over interior vertices (FP64 bits)
  unsigned long long m0;       // max |u| of the input (FP64 bits), never cleared
};

// Per-call fixed-point plan, recomputed identically by every CTA from the bounds.
struct Plan {
  bool fix;
  int Rf;  // scale of GF = 3/8 h^2 f
};

__device__ __forceinline__ double bits_to_d(unsigned long long b) { return __longlong_as_double((long long)b); }

__device__ __forceinline__ Plan make_plan(const SweepBounds *bnd, double g, int sweeps) {
  Plan p;
  const double M0 = bits_to_d(bnd->m0);
  const double gF = g * bits_to_d(bnd->fmax);
  // |u| after s sweeps <= M0 + 4 s g max|f|: every value of the call stays in range
  const double B = M0 + 4.0 * (double)(sweeps + 1) * gF;
  p.fix = fx::bound_ok(B) && fx::bound_ok(gF);
  p.Rf = gF > 0.0 ? fx::bound_exponent(gF) + 1 : -900;
  return p;
}

__device__ __forceinline__ int sweep_R(const SweepBounds *bnd, int slot, double g) {
  const double B = bits_to_d(bnd->umax[slot]) + 4.0 * g * bits_to_d(bnd->fmax);
  const int R = fx::bound_exponent(B) + 1;  // one spare bit: rounding can never reach 2^R
  return R < -900 ? -900 : R;
}

// Damping factor of the multi-sweep Jacobi kernels as an integer product: floor(D Wq /
// 2^62) with Wq = omega 2^62 rounded; for 0 < Wq < 2^62 it is the high word of
// D * (4 Wq) (unsigned high product, corrected for D < 0); Wq = 2^62 (omega = 1) is the
// identity.
struct Omega {
  unsigned long long w4;
  bool one;
  __device__ __forceinline__ Omega(long long Wq) : w4((unsigned long long)Wq << 2), one(Wq == (1ll << 62)) {}
  __device__ __forceinline__ long long operator()(long long D) const {
    const unsigned long long hi = __umul64hi((unsigned long long)D, w4) - (D < 0 ? w4 : 0ull);
    return one ? D : (long long)hi;
  }
};

// Arithmetic right shift by d (left shift for d < 0).
__device__ __forceinline__ long long shr_any(long long v, int d) {
  return d >= 63 ? (v >> 63) : (d >= 0 ? (v >> d) : (v << (-d)));
}

}  // namespace stencil
