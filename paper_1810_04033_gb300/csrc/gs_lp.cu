// Coloured Gauss-Seidel for reduced-precision storage (FP32, or bf16 storage with FP32
// arithmetic), the inner solver of the iterative refinement.  Same colour phases and
// two-launch out-of-place structure as the FP64 kernel (gs_fx.cu): the even launch
// updates rows A = (j even, k even) then B = (j odd, k even) of the even planes from
// X; the odd launch updates C = (j even, k odd) then D = (j odd, k odd) of the odd
// planes, reading the new even planes from Y.  In 3D, colours 2m and 2m+1 are
// uncoupled (Q1 face weight 0), so each phase updates whole x-rows; the result equals
// the sequential colour order.  Arithmetic is FP32 (u_new = 3/8 h^2 f + (2E + C)/32);
// bf16 values are widened on load and rounded to nearest even on every store.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

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

template <typename S>
__device__ void stage(float *slot, const S *plane, const Geo &q, int x0, int y0, bool odd_only) {
  const int nrows = odd_only ? LP_SH / 2 : LP_SH;
  for (int idx = threadIdx.x; idx < nrows * LP_SW; idx += LP_THREADS) {
    const int r = odd_only ? 2 * (idx >> 6) + 1 : (idx >> 6), col = idx & 63;
    const int64_t x = x0 - 2 + col, j = y0 - 2 + r;
    float v = 0.0f;
    if (plane && col < LP_TX + 4 && r < LP_TY + 4 && x >= 0 && x <= q.nx && j >= 0 && j <= q.ny)
      v = ld<S>(plane, j * q.pitch + x);
    slot[r * LP_SW + col] = v;
  }
}

template <typename S, int WHICH>
__device__ void lp_phase(const Geo &q, int x0, int y0, float *ce, const float *lo, const float *up,
                         const S *xplane, const S *fplane, S *yplane, float g) {
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
      v = quant<S>(fmaf(Pm + Pp + 2.0f * Q, 0.03125f, g * ld<S>(fplane, off)));
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
  bool have_lower = false;
  for (int64_t i = i0; i < i1; ++i) {
    const int64_t z = pz + 2 * i;
    const bool zin = z >= 1 && z < q.nz;
    if (zin) {
      if (!have_lower) stage<S>(slot(lo), N + (z - 1) * q.plane, q, x0, y0, false);
      stage<S>(slot(ce), X + z * q.plane, q, x0, y0, true);
      stage<S>(slot(up), N + (z + 1) * q.plane, q, x0, y0, false);
    } else if (z + 1 <= q.nz) {
      stage<S>(slot(up), N + (z + 1) * q.plane, q, x0, y0, false);
    }
    __syncthreads();
    if (zin) {
      lp_phase<S, 1>(q, x0, y0, slot(ce), slot(lo), slot(up), X + z * q.plane, f + z * q.plane,
                     Y + z * q.plane, g);
      __syncthreads();
      lp_phase<S, 2>(q, x0, y0, slot(ce), slot(lo), slot(up), X + z * q.plane, f + z * q.plane,
                     Y + z * q.plane, g);
    } else {
      for (int idx = threadIdx.x; idx < LP_TX * LP_TY; idx += LP_THREADS) {
        const int64_t x = x0 + idx % LP_TX, j = y0 + idx / LP_TX;
        if (x > q.nx || j > q.ny) continue;
        Y[z * q.plane + j * q.pitch + x] = X[z * q.plane + j * q.pitch + x];
      }
    }
    __syncthreads();
    const int t = lo;
    lo = up;
    up = t;
    have_lower = z + 1 <= q.nz;
  }
}

}  // namespace

template <typename S>
static cudaError_t gs_lp_sweeps(const Geo &q, S *u, const S *f, int sweeps, S *work, cudaStream_t s) {
  static bool attr = false;
  const size_t smem = 3 * (size_t)LP_PLANE * sizeof(float);
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_gs_lp_half<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const float g = (float)(0.375 * q.h * q.h);
  const unsigned tx = (unsigned)((q.nx + LP_TX) / LP_TX), ty = (unsigned)((q.ny + LP_TY) / LP_TY);
  if (ty > 65535) return cudaErrorInvalidConfiguration;
  S *X = u, *Y = work;
  for (int it = 0; it < sweeps; ++it) {
    for (int pz = 0; pz < 2; ++pz) {
      const int64_t ncentre = (q.nz - pz) / 2 + 1;
      const int cz = z_chunk((int64_t)tx * ty, ncentre, LP_CZ, 2, 8);
      const unsigned tz = (unsigned)((ncentre + cz - 1) / cz);
      k_gs_lp_half<S><<<dim3(tx, ty, tz), LP_THREADS, smem, s>>>(q, pz, X, pz == 0 ? X : Y, Y, f, g, cz);
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
