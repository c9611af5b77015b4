// Exact fixed-point arithmetic for FP64 stencil sums on the integer pipes.
//
// Why: on GB300 the FP64 pipe retires about 2 operations per clock per SM (FMA, ADD
// and every 64-bit conversion alike) while 32-bit integer adds retire about 111.  A
// 27-point update written in FP64 needs about 21 FP64 operations and is capped far
// below the memory roofline.  The Q1 stencil weights are small rationals (3D: 8/3,
// -1/6, -1/12; 2D: 8/3, -1/3; element matrix 12*K = {4, 0, -1}), so scaled by a
// common denominator they are integers.  Values are converted to int64 with FRAC
// fraction bits relative to a power-of-two bound 2^R on their magnitudes; the
// neighbour sums are then exact integer sums, and only the final scale-and-add runs on
// the FP64 pipe.  to_fixed and to_double use integer instructions only; to_double_cvt
// gives to_double's value through the FP64 pipe's conversion, for kernels whose integer
// pipe is the bottleneck while the FP64 pipe has room.
//
// Accuracy: each input is truncated to a multiple of 2^(R-FRAC) (|error| < 2^(R-52)),
// the integer sums are exact, and the conversion back rounds to nearest even; the
// result is accurate to a few units of 2^-52 relative to the bound, i.e. to the max
// norm of the data.  Subnormal inputs are read as zero; callers select the native FP64
// path when the bound is not finite or lies outside [2^-900, 2^1000].
#pragma once
#include <stdint.h>

namespace stencil {
namespace fx {

constexpr int FRAC = 52;

__host__ __device__ __forceinline__ unsigned long long dbits(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  __builtin_memcpy(&b, &x, 8);
  return b;
#endif
}

__host__ __device__ __forceinline__ double bitsd(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  __builtin_memcpy(&x, &b, 8);
  return x;
#endif
}

__host__ __device__ __forceinline__ int clz64(unsigned long long a) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)a);
#else
  return a ? __builtin_clzll(a) : 64;
#endif
}

// Bound exponent R with |x| < 2^R for all x <= b (b >= 0 finite); 0 for b == 0.
__host__ __device__ inline int bound_exponent(double b) {
  if (!(b > 0.0)) return 0;
  return (int)(dbits(b) >> 52) - 1022;  // b in [2^(e-1), 2^e)
}

// True when the fixed-point path may be used for data bounded by b.
__host__ __device__ inline bool bound_ok(double b) {
  return b == 0.0 || (b >= 0x1p-900 && b <= 0x1p+1000);
}

// x -> trunc(x * 2^(FRAC - R)) with rb = 1023 + R.  Requires |x| < 2^R.
__host__ __device__ __forceinline__ long long to_fixed(double x, int rb) {
  const unsigned long long b = dbits(x);
  const unsigned hi = (unsigned)(b >> 32);
  const int e = (int)((hi >> 20) & 0x7ffu);
  const int s = rb - e;  // >= 1; mantissa (53 bits incl. the hidden one) >> s
  const unsigned long long m = (b & 0x000fffffffffffffull) | 0x0010000000000000ull;
  const unsigned long long mag = s < 64 ? (m >> s) : 0ull;
  const long long sg = (long long)(int)hi >> 31;  // 0 or -1
  return ((long long)mag ^ sg) - sg;
}

// v * 2^e2, rounded to nearest even.  Requires the result (if v != 0) to be a normal
// double, which holds when 2^e2 >= 2^-1000 and |v| < 2^63.
__host__ __device__ __forceinline__ double to_double(long long v, int e2) {
  const long long sg = v >> 63;
  unsigned long long a = (unsigned long long)((v ^ sg) - sg);
  const int lz = clz64(a);               // 64 for a == 0
  a = lz < 64 ? (a << lz) : 0ull;        // leading one at bit 63
  unsigned long long mant = a >> 11;     // 53 bits incl. the leading one
  const unsigned rem = (unsigned)a & 0x7ffu;
  mant += (rem > 0x400u) | ((rem == 0x400u) & (unsigned)mant);
  // value = 1.f * 2^(63 - lz + e2); biased exponent minus one, then add the mantissa
  // (its leading one carries into the exponent field; a rounding overflow to 2^53
  // carries once more, which is exactly right)
  const long long ebm1 = (long long)(63 - lz + e2 + 1022);
  const unsigned long long bits =
      ((unsigned long long)ebm1 << 52) + mant + ((unsigned long long)sg & 0x8000000000000000ull);
  return a ? bitsd(bits) : 0.0;
}

// 2^e as a double, -1022 <= e <= 1023.
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

// The same value as to_double(v, e2), computed with the FP64 pipe's int64 -> double
// conversion (round to nearest even) and an exact power-of-two scaling: it moves the
// ~20 integer instructions of to_double off the integer pipe, which bounds the
// fixed-point kernels.  Requires -1022 <= e2 <= 1023 and a normal (or zero) result.
__device__ __forceinline__ double to_double_cvt(long long v, int e2) { return __ll2double_rn(v) * pow2d(e2); }

// |x| as ordered unsigned bits (monotone in |x| for finite and infinite x; NaN above).
__host__ __device__ __forceinline__ unsigned long long abs_bits(double x) {
  return dbits(x) & 0x7fffffffffffffffull;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

}  // namespace fx
}  // namespace stencil
