// Batches of cubic patches (regular patches of a block-structured mesh, Section 2):
// halo fill between neighbouring patches and coloured Gauss-Seidel sweeps of every
// patch in one persistent launch.
//
// Layout: patch p is a dense (n_p+1)^3 vertex array (x fastest) at element offset
// off_p of the packed buffers; its boundary shell is a halo refilled before every sweep
// from neighbour q = nbr[p][(dx+1) + 3 (dy+1) + 9 (dz+1)] (dir d = outward normal of
// the shell vertex; -1 = outer boundary, value 0).  Per axis the halo vertex takes the
// vertex of q nearest to its position (ties to the lower index), clamped into q's
// interior index range [1, n_q - 1].
//
// Sweep of one patch (one CTA): the 3D Q1 colour order (colour = x, y, z parities,
// ascending; colours 2m, 2m+1 uncoupled since face weights are 0) becomes 4 row phases
// A (j even, k even), B (j odd, k even), C (j even, k odd), D (j odd, k odd), executed
// as a wavefront over z: step t updates A and B of plane 2t, then C and D of plane
// 2t - 1.  Each value a phase reads is the one the sequential colour order would read,
// so the sweep runs in place.  Four planes (2t-2 .. 2t+1) sit in shared memory as
// exact int64 fixed point (fixed.cuh) relative to a per-patch bound: max |u| of the
// patch (tracked from the previous sweep and the halo fill) plus 4 (3/8) h^2 max |f|.
// CTAs take patches from a work counter, largest first.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "fixed.cuh"
#include "internal.h"

namespace stencil {
namespace {

constexpr int P_MAXN = 64;

struct PatchDev {
  int n;
  int pad;
  int64_t off;
  double h;
};

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}

__device__ unsigned long long block_max_u64(unsigned long long v, unsigned long long *red) {
  v = fx::warp_max_u64(v);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  unsigned long long m = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = umax64(m, red[k]);
  return m;
}

// max |u| over the whole patch and max |f| over its interior, one CTA per patch
__global__ void k_patch_prep(const PatchDev *pd, int npatch, const double *u, const double *f,
                             unsigned long long *umax, unsigned long long *fmx) {
  __shared__ unsigned long long red[32];
  for (int p = blockIdx.x; p < npatch; p += gridDim.x) {
    const int n = pd[p].n, W = n + 1;
    const int64_t off = pd[p].off;
    unsigned long long mu = 0, mf = 0;
    for (int idx = threadIdx.x; idx < W * W * W; idx += blockDim.x) {
      const int i = idx % W, j = (idx / W) % W, k = idx / (W * W);
      mu = umax64(mu, fx::abs_bits(u[off + idx]));
      if (i > 0 && i < n && j > 0 && j < n && k > 0 && k < n) mf = umax64(mf, fx::abs_bits(f[off + idx]));
    }
    mu = block_max_u64(mu, red);
    mf = block_max_u64(mf, red);
    if (threadIdx.x == 0) {
      umax[p] = mu;
      fmx[p] = mf;
    }
  }
}

// halo index on one axis (see header)
__device__ __forceinline__ int halo_index(int idx, int d, int n, int m) {
  const int num = (idx - d * n) * m;  // >= 0
  int t = (2 * num + n - 1) / (2 * n);
  return t < 1 ? 1 : (t > m - 1 ? m - 1 : t);
}

// One CTA per patch (grid-stride).  The 26 neighbour entries (id, edge, offset) are
// read into shared memory once; then the block's threads run over the whole shell as one
// index space (the two z faces, the two y faces without their z edges, the two x faces
// without their y and z edges), each vertex finding its outward direction from its
// indices, so that every thread has work whatever the direction.
__global__ void k_patch_halo(const PatchDev *pd, const int *nbr, int npatch, double *u,
                             unsigned long long *hmax) {
  __shared__ unsigned long long red[32];
  __shared__ int s_m[27];
  __shared__ long long s_off[27];
  for (int p = blockIdx.x; p < npatch; p += gridDim.x) {
    const int n = pd[p].n, W = n + 1, P = W * W;
    const int64_t off = pd[p].off;
    if (threadIdx.x < 27) {
      const int q = threadIdx.x == 13 ? -1 : nbr[27 * p + threadIdx.x];
      s_m[threadIdx.x] = q >= 0 ? pd[q].n : -1;
      s_off[threadIdx.x] = q >= 0 ? pd[q].off : 0;
    }
    __syncthreads();
    unsigned long long mh = 0;
    const int nA = 2 * P, nB = 2 * W * (n - 1), nC = 2 * (n - 1) * (n - 1);
    for (int t = threadIdx.x; t < nA + nB + nC; t += blockDim.x) {
      int i, j, k;
      if (t < nA) {  // z = 0 and z = n, whole planes
        k = t < P ? 0 : n;
        const int r = t < P ? t : t - P;
        j = r / W;
        i = r - j * W;
      } else if (t < nA + nB) {  // y = 0 and y = n, z = 1 .. n-1
        const int r = t - nA, zz = r / (2 * W), rr = r - zz * 2 * W;
        k = 1 + zz;
        j = rr < W ? 0 : n;
        i = rr < W ? rr : rr - W;
      } else {  // x = 0 and x = n, y and z = 1 .. n-1
        const int r = t - nA - nB, zz = r / (2 * (n - 1)), rr = r - zz * 2 * (n - 1);
        k = 1 + zz;
        j = 1 + (rr >> 1);
        i = (rr & 1) ? n : 0;
      }
      const int dx = i == 0 ? -1 : (i == n ? 1 : 0), dy = j == 0 ? -1 : (j == n ? 1 : 0),
                dz = k == 0 ? -1 : (k == n ? 1 : 0);
      const int dir = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
      const int m = s_m[dir];
      double v = 0.0;
      if (m >= 0) {
        const int iq = halo_index(i, dx, n, m), jq = halo_index(j, dy, n, m), kq = halo_index(k, dz, n, m);
        v = u[s_off[dir] + ((int64_t)kq * (m + 1) + jq) * (m + 1) + iq];
      }
      u[off + ((int64_t)k * W + j) * W + i] = v;
      mh = umax64(mh, fx::abs_bits(v));
    }
    mh = block_max_u64(mh, red);  // its barriers also keep s_m / s_off until every thread is done
    if (threadIdx.x == 0) hmax[p] = mh;
  }
}

template <bool FIX>
__device__ __forceinline__ long long enc(double v, int rb) {
  if (FIX) return fx::to_fixed(v, rb);
  return __double_as_longlong(v);
}

template <bool FIX>
__device__ __forceinline__ long long add(long long a, long long b) {
  if (FIX) return a + b;
  return __double_as_longlong(__longlong_as_double(a) + __longlong_as_double(b));
}

// Software pipeline of one patch sweep: the next step's two planes are copied from
// global memory into their shared-memory slots by cp.async while the current step
// computes (six slots: four planes in use, two arriving), and converted to fixed point
// in place when the step starts; the right-hand side of a thread's first item of each
// phase (P_FPF) is loaded when the step starts, the rest inside the phase.
constexpr int P_SLOTS = 6;
constexpr int P_FPF = 1;

__device__ __forceinline__ long long *patch_slot(long long *smem, int P, int z) { return smem + (z % P_SLOTS) * P; }

// Start copying planes z0 and z0 + 1 (those <= n) into their slots, raw FP64 bits; one
// commit group.
__device__ __forceinline__ void stage_async(long long *smem, const double *u, int P, int z0, int n) {
  for (int idx = threadIdx.x; idx < 2 * P; idx += blockDim.x) {
    const int up = idx >= P, z = z0 + up, e = idx - (up ? P : 0);
    if (z <= n) {
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(patch_slot(smem, P, z) + e);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(u + (int64_t)z * P + e) : "memory");
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// Wait for this thread's copies of planes z0, z0 + 1 and convert them in place (the
// same element mapping as stage_async, so every thread converts what it copied).
template <bool FIX>
__device__ __forceinline__ void stage_convert(long long *smem, int P, int z0, int n, int rb) {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (!FIX) return;
  for (int idx = threadIdx.x; idx < 2 * P; idx += blockDim.x) {
    const int up = idx >= P, z = z0 + up, e = idx - (up ? P : 0);
    if (z <= n) {
      long long *v = patch_slot(smem, P, z) + e;
      *v = enc<true>(__longlong_as_double(*v), rb);
    }
  }
}

// right-hand sides of this thread's first P_FPF items of a phase (rows of parity pr)
__device__ __forceinline__ void phase_f(double (&fv)[P_FPF], const double *fplane, int n, int pr) {
  const int W = n + 1;
  const int j0 = pr ? 1 : 2;
  const int nrows = n - 1 >= j0 ? (n - 1 - j0) / 2 + 1 : 0;
  const int items = nrows * (n - 1);
#pragma unroll
  for (int k = 0; k < P_FPF; ++k) {
    const int it = threadIdx.x + k * (int)blockDim.x;
    fv[k] = fplane && it < items ? fplane[(j0 + 2 * (it / (n - 1))) * W + 1 + it % (n - 1)] : 0.0;
  }
}

// rows of parity pr of plane z (interior), from planes z-1, z, z+1 in shared memory
template <bool FIX>
__device__ void patch_phase(long long *ce, const long long *lo, const long long *up, int n, int pr,
                            const double *fplane, const double (&fv)[P_FPF], double *uplane, double g, int rb,
                            int e2, unsigned long long &vmax) {
  const int W = n + 1, nm1 = n - 1;
  const int j0 = pr ? 1 : 2;  // first interior row of parity pr
  const int nrows = n - 1 >= j0 ? (n - 1 - j0) / 2 + 1 : 0;
  const int items = nrows * nm1;
  // item it is (row it / nm1, column it % nm1); the thread's items advance by blockDim,
  // so row and column advance by fixed steps (no division per item)
  int r = (int)threadIdx.x / nm1, cc = (int)threadIdx.x - r * nm1;
  const int dr = (int)blockDim.x / nm1, dc = (int)blockDim.x - dr * nm1;
  int k = 0;
  for (int it = threadIdx.x; it < items; it += blockDim.x, ++k) {
    const int j = j0 + 2 * r, i = 1 + cc;
    cc += dc;
    r += dr;
    if (cc >= nm1) {
      cc -= nm1;
      ++r;
    }
    const int c = j * W + i;
    // E: edges (x,y in plane; x,z; y,z), C: corners; face weights are 0
    const long long Exy = add<FIX>(add<FIX>(ce[c - W - 1], ce[c - W + 1]), add<FIX>(ce[c + W - 1], ce[c + W + 1]));
    const long long Exz = add<FIX>(add<FIX>(lo[c - 1], lo[c + 1]), add<FIX>(up[c - 1], up[c + 1]));
    const long long Eyz = add<FIX>(add<FIX>(lo[c - W], lo[c + W]), add<FIX>(up[c - W], up[c + W]));
    const long long C = add<FIX>(add<FIX>(add<FIX>(lo[c - W - 1], lo[c - W + 1]), add<FIX>(lo[c + W - 1], lo[c + W + 1])),
                                 add<FIX>(add<FIX>(up[c - W - 1], up[c - W + 1]), add<FIX>(up[c + W - 1], up[c + W + 1])));
    const long long E = add<FIX>(add<FIX>(Exy, Exz), Eyz);
    const long long S = add<FIX>(add<FIX>(E, E), C);  // 2E + C
    double f0 = 0.0;
#pragma unroll
    for (int q = 0; q < P_FPF; ++q)
      if (k == q) f0 = fv[q];
    const double fval = k < P_FPF ? f0 : fplane[c];
    double un;
    if (FIX)
      un = fma(g, fval, fx::to_double(S, e2));
    else
      un = fma(__longlong_as_double(S), 0.03125, g * fval);
    ce[c] = enc<FIX>(un, rb);
    uplane[c] = un;
    vmax = umax64(vmax, fx::abs_bits(un));
  }
}

template <bool FIX>
__device__ void patch_sweep(int n, double *u, const double *f, double g, int R, long long *smem,
                            unsigned long long &vmax) {
  const int W = n + 1, P = W * W;
  const int rb = 1023 + R, e2 = R - fx::FRAC - 5;
  auto slot = [&](int z) -> long long * { return patch_slot(smem, P, z); };
  stage_async(smem, u, P, 0, n);
  for (int t = 0; 2 * t - 1 <= n; ++t) {
    const int za = 2 * t, zc = 2 * t - 1;
    // planes za, za+1 arrived (issued one step ago); the next two go into the slots of
    // za-4, za-3, which the previous step was the last to read
    if (za <= n) stage_convert<FIX>(smem, P, za, n, rb);
    if (za + 2 <= n) stage_async(smem, u, P, za + 2, n);
    const bool da = za >= 1 && za <= n - 1, dc = zc >= 1 && zc <= n - 1;
    double fa0[P_FPF], fa1[P_FPF], fc0[P_FPF], fc1[P_FPF];
    phase_f(fa0, da ? f + (int64_t)za * P : nullptr, n, 0);
    phase_f(fa1, da ? f + (int64_t)za * P : nullptr, n, 1);
    phase_f(fc0, dc ? f + (int64_t)zc * P : nullptr, n, 0);
    phase_f(fc1, dc ? f + (int64_t)zc * P : nullptr, n, 1);
    __syncthreads();
    if (da) {
      patch_phase<FIX>(slot(za), slot(za - 1), slot(za + 1), n, 0, f + (int64_t)za * P, fa0, u + (int64_t)za * P,
                       g, rb, e2, vmax);
      __syncthreads();
      patch_phase<FIX>(slot(za), slot(za - 1), slot(za + 1), n, 1, f + (int64_t)za * P, fa1, u + (int64_t)za * P,
                       g, rb, e2, vmax);
      __syncthreads();
    }
    if (dc) {
      patch_phase<FIX>(slot(zc), slot(zc - 1), slot(zc + 1), n, 0, f + (int64_t)zc * P, fc0, u + (int64_t)zc * P,
                       g, rb, e2, vmax);
      __syncthreads();
      patch_phase<FIX>(slot(zc), slot(zc - 1), slot(zc + 1), n, 1, f + (int64_t)zc * P, fc1, u + (int64_t)zc * P,
                       g, rb, e2, vmax);
    }
    __syncthreads();
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");  // nothing in flight when the CTA moves on
}

__global__ void __launch_bounds__(512) k_patch_gs(const PatchDev *pd, const int *order, int npatch, double *u, const double *f,
                           unsigned long long *umax, const unsigned long long *hmax,
                           const unsigned long long *fmx, unsigned *counter) {
  extern __shared__ long long psm[];
  __shared__ unsigned long long red[32];
  __shared__ int cur;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned w = atomicAdd(counter, 1u);
      cur = w < (unsigned)npatch ? order[w] : -1;
    }
    __syncthreads();
    const int p = cur;
    if (p < 0) return;
    const int n = pd[p].n;
    const double h = pd[p].h, g = 0.375 * h * h;
    const double M = fmax(__longlong_as_double((long long)umax[p]), __longlong_as_double((long long)hmax[p]));
    const double B = M + 4.0 * g * __longlong_as_double((long long)fmx[p]);
    const int R = fx::bound_exponent(B) + 1;
    unsigned long long vmax = 0;
    double *up = u + pd[p].off;
    const double *fp = f + pd[p].off;
    if (fx::bound_ok(B))
      patch_sweep<true>(n, up, fp, g, R, psm, vmax);
    else
      patch_sweep<false>(n, up, fp, g, R, psm, vmax);
    vmax = block_max_u64(vmax, red);
    if (threadIdx.x == 0) umax[p] = umax64(vmax, hmax[p]);
    __syncthreads();  // cur is rewritten by the next claim
  }
}

}  // namespace
}  // namespace stencil

using namespace stencil;

struct stencil_batch {
  int npatch = 0;
  int maxn = 0;
  int64_t span = 0;        // elements covered by the packed arrays
  int device = 0;
  stencil::PatchDev *d_pd = nullptr;
  int *d_nbr = nullptr;
  int *d_order = nullptr;
  unsigned long long *d_bounds = nullptr;  // umax, hmax, fmax (npatch each)
  unsigned *d_counters = nullptr;
  int ncounters = 0;
  int threads = 256;       // launch shape (autotuned)
  int ctas_per_sm = 4;
  int64_t interior_updates = 0;
};

static size_t patch_smem(int maxn) { return P_SLOTS * (size_t)(maxn + 1) * (maxn + 1) * sizeof(long long); }

// The shared-memory limit of k_patch_gs is a per-device kernel attribute, while each
// batch needs its own amount (it grows with the largest patch).  The limit is only ever
// raised, so a batch created later with smaller patches cannot lower it under a batch
// that needs more; a launch still asks for exactly its own amount.
static cudaError_t raise_patch_smem_limit(size_t bytes) {
  static std::mutex mu;
  static size_t limit[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaFuncSetAttribute(k_patch_gs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  std::lock_guard<std::mutex> lk(mu);
  if (bytes <= limit[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(k_patch_gs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) limit[dev] = bytes;
  return e;
}

extern "C" {

int stencil_patch_batch_create(const stencil_patch_desc_t *patches, int32_t npatch, const int32_t *neighbours,
                               stencil_batch_t **out) {
  if (!out) return set_error(STENCIL_EINVAL, "patch_batch_create: out is NULL");
  *out = nullptr;
  if (!patches || !neighbours || npatch < 1) return set_error(STENCIL_EINVAL, "patch_batch_create: empty batch");
  std::vector<PatchDev> pd(npatch);
  int maxn = 0;
  int64_t span = 0, upd = 0;
  for (int p = 0; p < npatch; ++p) {
    const int n = patches[p].n;
    if (n < 2 || n > P_MAXN) return set_error(STENCIL_EINVAL, "patch_batch_create: n must be in [2, 64]");
    if (patches[p].offset < 0) return set_error(STENCIL_EINVAL, "patch_batch_create: negative offset");
    const double h = patches[p].h > 0.0 ? patches[p].h : 1.0 / n;
    pd[p] = PatchDev{n, 0, patches[p].offset, h};
    maxn = std::max(maxn, n);
    span = std::max(span, patches[p].offset + (int64_t)(n + 1) * (n + 1) * (n + 1));
    upd += (int64_t)(n - 1) * (n - 1) * (n - 1);
  }
  for (int64_t k = 0; k < 27LL * npatch; ++k)
    if (neighbours[k] < -1 || neighbours[k] >= npatch)
      return set_error(STENCIL_EINVAL, "patch_batch_create: neighbour index out of range");
  std::vector<int> order(npatch);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pd[a].n > pd[b].n; });
  stencil_batch *b = new stencil_batch();
  b->npatch = npatch;
  b->maxn = maxn;
  b->span = span;
  b->interior_updates = upd;
  cudaGetDevice(&b->device);
  bool ok = cudaMalloc(&b->d_pd, npatch * sizeof(PatchDev)) == cudaSuccess &&
            cudaMalloc(&b->d_nbr, 27 * (size_t)npatch * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&b->d_order, npatch * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&b->d_bounds, 3 * (size_t)npatch * sizeof(unsigned long long)) == cudaSuccess;
  ok = ok && cudaMemcpy(b->d_pd, pd.data(), npatch * sizeof(PatchDev), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(b->d_nbr, neighbours, 27 * (size_t)npatch * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(b->d_order, order.data(), npatch * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
  const size_t smem = patch_smem(maxn);
  ok = ok && raise_patch_smem_limit(smem) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    stencil_patch_batch_destroy(b);
    return set_error(STENCIL_ENOMEM, "patch_batch_create: device allocation failed");
  }
  *out = b;
  return STENCIL_OK;
}

int stencil_patch_batch_destroy(stencil_batch_t *b) {
  if (!b) return STENCIL_OK;
  cudaFree(b->d_pd);
  cudaFree(b->d_nbr);
  cudaFree(b->d_order);
  cudaFree(b->d_bounds);
  cudaFree(b->d_counters);
  delete b;
  return STENCIL_OK;
}

static int batch_sweeps(stencil_batch_t *b, double *u, const double *f, int sweeps, cudaStream_t s, int threads,
                        int ctas_per_sm) {
  if (sweeps > b->ncounters) {
    cudaFree(b->d_counters);
    b->d_counters = nullptr;
    const int nc = std::max(sweeps, 64);
    if (cudaMalloc(&b->d_counters, nc * sizeof(unsigned)) != cudaSuccess) {
      b->ncounters = 0;
      return set_error(STENCIL_ENOMEM, "patch_batch_smooth: counter allocation failed");
    }
    b->ncounters = nc;
  }
  unsigned long long *umax = b->d_bounds, *hmax = umax + b->npatch, *fmax = hmax + b->npatch;
  cudaError_t e = cudaMemsetAsync(b->d_counters, 0, sweeps * sizeof(unsigned), s);
  if (e) return set_error(STENCIL_ECUDA, std::string("patch_batch_smooth: ") + cudaGetErrorString(e));
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  const unsigned gridp = (unsigned)std::min(b->npatch, sms * 8);
  k_patch_prep<<<gridp, 256, 0, s>>>(b->d_pd, b->npatch, u, f, umax, fmax);
  const size_t smem = patch_smem(b->maxn);
  const unsigned grid = (unsigned)std::min(b->npatch, sms * ctas_per_sm);
  for (int it = 0; it < sweeps; ++it) {
    k_patch_halo<<<gridp, 256, 0, s>>>(b->d_pd, b->d_nbr, b->npatch, u, hmax);
    k_patch_gs<<<grid, threads, smem, s>>>(b->d_pd, b->d_order, b->npatch, u, f, umax, hmax, fmax,
                                            b->d_counters + it);
  }
  e = cudaGetLastError();
  if (e) return set_error(STENCIL_ECUDA, std::string("patch_batch_smooth: ") + cudaGetErrorString(e));
  return STENCIL_OK;
}

int stencil_patch_batch_smooth(stencil_batch_t *b, double *u_all, const double *f_all, int sweeps, void *stream) {
  if (!b) return set_error(STENCIL_EINVAL, "patch_batch_smooth: batch is NULL");
  if (!u_all || !f_all || (uintptr_t)u_all % 8 || (uintptr_t)f_all % 8)
    return set_error(STENCIL_EINVAL, "patch_batch_smooth: u_all/f_all NULL or misaligned");
  if (sweeps < 0) return set_error(STENCIL_EINVAL, "patch_batch_smooth: sweeps < 0");
  if (sweeps == 0) return STENCIL_OK;
  return batch_sweeps(b, u_all, f_all, sweeps, (cudaStream_t)stream, b->threads, b->ctas_per_sm);
}

int stencil_patch_batch_autotune(stencil_batch_t *b, const double *u_all, const double *f_all, void *stream) {
  if (!b || !u_all || !f_all) return set_error(STENCIL_EINVAL, "patch_batch_autotune: NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  double *tmp = nullptr;
  if (cudaMalloc(&tmp, (size_t)b->span * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return set_error(STENCIL_ENOMEM, "patch_batch_autotune: scratch allocation failed");
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int th[] = {128, 256, 512};
  const int cps[] = {2, 4, 8};
  int smem_sm = 0;  // shared memory per SM; each resident CTA also reserves 1 KB
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, b->device);
  float best = 1e30f;
  int bt = b->threads, bc = b->ctas_per_sm;
  int rc = STENCIL_OK;
  for (int t : th) {
    for (int c : cps) {
      if ((patch_smem(b->maxn) + 1024) * c > (size_t)smem_sm) continue;  // does not fit on an SM
      cudaMemcpyAsync(tmp, u_all, (size_t)b->span * sizeof(double), cudaMemcpyDeviceToDevice, s);
      rc = batch_sweeps(b, tmp, f_all, 1, s, t, c);  // warm
      if (rc) break;
      cudaEventRecord(e0, s);
      rc = batch_sweeps(b, tmp, f_all, 3, s, t, c);
      cudaEventRecord(e1, s);
      if (rc) break;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bt = t;
        bc = c;
      }
    }
    if (rc) break;
  }
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(tmp);
  if (rc) return rc;
  b->threads = bt;
  b->ctas_per_sm = bc;
  return STENCIL_OK;
}

int stencil_patch_batch_config(const stencil_batch_t *b, int32_t *threads, int32_t *ctas_per_sm) {
  if (!b) return set_error(STENCIL_EINVAL, "patch_batch_config: batch is NULL");
  if (threads) *threads = b->threads;
  if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
  return STENCIL_OK;
}

}  // extern "C"
