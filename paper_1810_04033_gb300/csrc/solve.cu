// Mixed-precision iterative refinement (stencil_solve) and the correction update.
//
// Outer iteration, starting from the FP64 iterate x (its boundary holds the Dirichlet
// data): r = f - A x in FP64 with ||r||, ||f|| in FP64 (fixed-order reduction); stop when
// ||r|| / ||f|| <= rel_tol; round r to the inner type (FP32; bf16 via FP32); from e = 0
// run `inner_sweeps` coloured Gauss-Seidel sweeps on A e = r in the inner precision;
// x += e widened exactly to FP64.  With inner type FP64 the inner sweeps are the FP64
// smoother itself.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>

#include "internal.h"

namespace stencil {
namespace {

template <typename E>
__device__ __forceinline__ double widen(E v);
template <>
__device__ __forceinline__ double widen<double>(double v) {
  return v;
}
template <>
__device__ __forceinline__ double widen<float>(float v) {
  return (double)v;
}
template <>
__device__ __forceinline__ double widen<__nv_bfloat16>(__nv_bfloat16 v) {
  return (double)__bfloat162float(v);
}

template <typename E>
__global__ void __launch_bounds__(256) k_add_correction(Geo q, int dim, double *__restrict__ x,
                                                        const E *__restrict__ e) {
  const int64_t nrows = (q.nz + 1) * (q.ny + 1);
  for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int64_t k = row / (q.ny + 1), j = row % (q.ny + 1);
    if (j == 0 || j == q.ny || (dim == 3 && (k == 0 || k == q.nz))) continue;
    const int64_t base = k * q.plane + j * q.pitch;
    for (int64_t i = 1 + threadIdx.x; i < q.nx; i += blockDim.x) x[base + i] += widen<E>(e[base + i]);
  }
}

}  // namespace

cudaError_t launch_add_correction(const Geo &q, int dim, double *x, const void *e, int dtype, cudaStream_t s) {
  const int64_t nrows = (q.nz + 1) * (q.ny + 1);
  const unsigned nb = (unsigned)(nrows < 4864 ? nrows : 4864);
  if (dtype == STENCIL_F64)
    k_add_correction<double><<<nb, 256, 0, s>>>(q, dim, x, (const double *)e);
  else if (dtype == STENCIL_F32)
    k_add_correction<float><<<nb, 256, 0, s>>>(q, dim, x, (const float *)e);
  else
    k_add_correction<__nv_bfloat16><<<nb, 256, 0, s>>>(q, dim, x, (const __nv_bfloat16 *)e);
  return cudaGetLastError();
}

}  // namespace stencil
