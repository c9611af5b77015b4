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
