// Allocation-free residual and norms (stencil_residual_noalloc).
//
// stencil_residual keeps its reduction scratch in device memory that the library
// allocates with cudaMalloc on first use.  Some callers cannot let a library allocate:
// cudaMalloc and cudaFree can synchronise the whole device, which a latency-bound
// loop keeping several streams busy cannot afford; another allocator (a framework's
// caching pool) may already hold nearly all device memory, so a raw cudaMalloc fails
// even though the caller has room in its own pool; and some deployments forbid any
// device allocation after start-up.  This entry point computes the same residual and
// norms with its scratch in a fixed array that lives in the library's device image,
// so the call itself allocates nothing.
//
// Limit: the array holds the per-CTA partial sums of at most kNoAllocMaxBlocks CTAs,
// each summing kNoAllocRowsPerBlock x-rows, i.e. grids of at most
// kNoAllocMaxBlocks * kNoAllocRowsPerBlock = 524288 rows ((n_z+1)*(n_y+1) in 3D,
// n_y+1 in 2D); larger grids are rejected with STENCIL_EINVAL.  The array costs
// 128 KiB of device memory on every GPU that loads the library, until the process
// exits.  All calls share it: calls whose kernels overlap on the GPU (different
// streams, or threads without ordering) race on it and must be serialised by the
// caller.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace stencil {
int check_grid(const stencil_grid_t *g);  // api.cu

namespace {

constexpr int kNoAllocMaxBlocks = 8192;
constexpr int kNoAllocRowsPerBlock = 64;
constexpr int kNoAllocThreads = 256;

struct NoAllocScratch {
  double partials[2 * kNoAllocMaxBlocks];  // (sum r^2, sum f^2) per CTA
  unsigned int counter;                    // CTAs finished; zeroed before each launch
};

// The scratch: part of the library's device image, one copy per device.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

__device__ __forceinline__ double edge_corner_sum_weighted(const double *__restrict__ c,
                                                           int64_t P, int64_t Z) {
  const double E = ((c[-1 - P] + c[1 - P]) + (c[-1 + P] + c[1 + P])) +
                   ((c[-1 - Z] + c[1 - Z]) + (c[-1 + Z] + c[1 + Z])) +
                   ((c[-P - Z] + c[P - Z]) + (c[-P + Z] + c[P + Z]));
  const double C = ((c[-1 - P - Z] + c[1 - P - Z]) + (c[-1 + P - Z] + c[1 + P - Z])) +
                   ((c[-1 - P + Z] + c[1 - P + Z]) + (c[-1 + P + Z] + c[1 + P + Z]));
  return fma(2.0, E, C);  // 2E + C
}

__device__ __forceinline__ double ring8(const double *__restrict__ c, int64_t P) {
  return ((c[-1 - P] + c[-P]) + (c[1 - P] + c[-1])) + ((c[1] + c[-1 + P]) + (c[P] + c[1 + P]));
}

__device__ __forceinline__ void cta_sum2(double &a, double &b, double *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sh[2 * w] = a;
    sh[2 * w + 1] = b;
  }
  __syncthreads();
  if (w == 0) {
    constexpr int NW = kNoAllocThreads / 32;
    a = l < NW ? sh[2 * l] : 0.0;
    b = l < NW ? sh[2 * l + 1] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
  }
}

// CTA b sums the contiguous rows [b*R, (b+1)*R); the last CTA to finish adds the
// partials in a fixed order (a strided subset per thread, then a fixed shuffle tree),
// so the result depends only on the input and the grid.
__global__ void __launch_bounds__(kNoAllocThreads)
    k_residual_noalloc(Geo q, int dim, const double *__restrict__ u, const double *__restrict__ f,
                       double *__restrict__ r, double *norms2, NoAllocScratch *scr, double inv_h2) {
  __shared__ double sh[2 * kNoAllocThreads / 32];
  __shared__ bool last;
  double rr = 0.0, ff = 0.0;
  const int64_t nrows = (q.nz + 1) * (q.ny + 1);
  const int64_t row0 = (int64_t)blockIdx.x * kNoAllocRowsPerBlock;
  const int64_t row1 = row0 + kNoAllocRowsPerBlock < nrows ? row0 + kNoAllocRowsPerBlock : nrows;
  for (int64_t row = row0; row < row1; ++row) {
    const int64_t k = row / (q.ny + 1), j = row % (q.ny + 1);
    const bool row_inner = j > 0 && j < q.ny && (dim == 2 || (k > 0 && k < q.nz));
    for (int64_t i = threadIdx.x; i <= q.nx; i += blockDim.x) {
      const int64_t p = k * q.plane + j * q.pitch + i;
      if (!row_inner || i == 0 || i == q.nx) {
        if (r) r[p] = 0.0;
        continue;
      }
      // 3D: 12 S u = 32 u - (2E + C);  2D: 3 S u = 8 u - N
      const double Su = dim == 3 ? fma(32.0, u[p], -edge_corner_sum_weighted(u + p, q.pitch, q.plane)) *
                                       (1.0 / 12.0)
                                 : fma(8.0, u[p], -ring8(u + p, q.pitch)) * (1.0 / 3.0);
      const double fp = f[p];
      const double rp = fma(-Su, inv_h2, fp);
      if (r) r[p] = rp;
      rr = fma(rp, rp, rr);
      ff = fma(fp, fp, ff);
    }
  }
  cta_sum2(rr, ff, sh);
  if (threadIdx.x == 0) {
    scr->partials[2 * blockIdx.x] = rr;
    scr->partials[2 * blockIdx.x + 1] = ff;
    __threadfence();
    last = atomicAdd(&scr->counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double a = 0.0, b = 0.0;
  for (int t = threadIdx.x; t < (int)gridDim.x; t += blockDim.x) {
    a += __ldcg(scr->partials + 2 * t);
    b += __ldcg(scr->partials + 2 * t + 1);
  }
  __syncthreads();
  cta_sum2(a, b, sh);
  if (threadIdx.x == 0) {
    norms2[0] = a;
    norms2[1] = b;
  }
}

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
NoAllocScratch *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device, looked up once per device
// (in host code the symbol name is only a host-side handle, not a device address).
int scratch_address(NoAllocScratch **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(STENCIL_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(STENCIL_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_error(STENCIL_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = (NoAllocScratch *)p;
  }
  *out = g_scratch_addr[dev];
  return STENCIL_OK;
}

bool overlaps(const void *a, const void *b, size_t bytes) {
  const char *x = (const char *)a, *y = (const char *)b;
  return x < y + bytes && y < x + bytes;
}

}  // namespace
}  // namespace stencil

using namespace stencil;

extern "C" int stencil_residual_noalloc(const stencil_grid_t *g, const void *u, const void *f,
                                        void *r, double *d_norms2, void *stream) {
  int rc = check_grid(g);
  if (rc) return rc;
  if (g->dtype != STENCIL_F64) return set_error(STENCIL_EINVAL, "residual_noalloc supports F64 only");
  if (g->op != STENCIL_OP_Q1) return set_error(STENCIL_EINVAL, "residual_noalloc: the Q1 operator only");
  if (!u || !f || !d_norms2) return set_error(STENCIL_EINVAL, "u, f and d_norms2 must not be NULL");
  if ((uintptr_t)u % 8 || (uintptr_t)f % 8 || (uintptr_t)d_norms2 % 8 || (r && (uintptr_t)r % 8))
    return set_error(STENCIL_EINVAL, "arrays must be 8-byte aligned");
  const Geo q = make_geo(*g);
  const int64_t nrows = (q.nz + 1) * (q.ny + 1);
  const int64_t blocks = (nrows + kNoAllocRowsPerBlock - 1) / kNoAllocRowsPerBlock;
  if (blocks > kNoAllocMaxBlocks)
    return set_error(STENCIL_EINVAL,
                     "grid too large for the allocation-free residual: " + std::to_string(nrows) +
                         " x-rows, at most " +
                         std::to_string((int64_t)kNoAllocMaxBlocks * kNoAllocRowsPerBlock) +
                         " supported (use stencil_residual)");
  const size_t bytes = (size_t)span_elems(q) * 8;
  if (r && (overlaps(r, u, bytes) || overlaps(r, f, bytes)))
    return set_error(STENCIL_EINVAL, "r overlaps u or f");
  NoAllocScratch *scr = nullptr;
  if ((rc = scratch_address(&scr))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  // the counter keeps the previous call's final value: clear it on this stream
  cudaError_t e = cudaMemsetAsync(&scr->counter, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return set_error(STENCIL_ECUDA, std::string("residual_noalloc: ") + cudaGetErrorString(e));
  k_residual_noalloc<<<(unsigned)blocks, kNoAllocThreads, 0, s>>>(
      q, g->dim, (const double *)u, (const double *)f, (double *)r, d_norms2, scr, 1.0 / (q.h * q.h));
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(STENCIL_ECUDA, std::string("residual_noalloc: ") + cudaGetErrorString(e));
  return STENCIL_OK;
}
