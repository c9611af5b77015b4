// Dependency-driven red-black sweeps: the GPU form of the paper's Hyb-depend variant
// (Section 5, Algorithm 1): tasks carry their data dependencies, and are issued in the
// order the colouring prescribes, so that a task rarely has to wait.
//
// The grid (5/7-point finite differences, red-black, fd.cu) is cut into blocks: in 2D
// `rows` x-rows, in 3D `rows` z-planes by `cols` y-rows.  Task (p, b) applies colour
// phase p of the whole run (p = 2 s + c: sweep s, colour c; colour 0 = the
// (i+j+k)-odd vertices, colour 1 = the even ones) to block b, in place.  It reads only
// the other colour, in b and its face-neighbour blocks, which phase p-1 wrote; and it
// overwrites values that phase p-1 read in those blocks.  So task (p, b) may start once
// b and its face neighbours (2D: b +- 1; 3D: +-1 in z and in y) have finished phase p-1,
// and no other ordering is needed: no grid-wide barrier between colours or sweeps.
//
// One persistent cooperative launch (all CTAs co-resident) claims tasks from an atomic
// counter in phase-major order (every block of phase p before any of phase p+1: the
// colour order as issue hint).  done[b] counts the phases finished on block b; a task
// waits (one thread, acquire loads, bounded by a time limit) until its three
// neighbours reached p, computes, and publishes done[b] = p + 1 with a release store.
// Because tasks are claimed in an order consistent with the dependencies and every
// claimed task belongs to a running CTA, a wait always ends unless something else
// failed; the time limit turns such a failure into STENCIL_ETIMEDOUT (an error flag
// that every CTA polls) instead of a hang.  Data written by other CTAs during the
// launch is read through L2 (ld.global.cg).
#include <cuda_runtime.h>
#include <stdint.h>

#include "cost.cuh"
#include "internal.h"

namespace stencil {
namespace {

constexpr int D_THREADS = 256;

struct DepState {
  unsigned long long next_task;  // claim counter
  int error;                     // 1: a wait timed out
  int stalled_at;                // the block a timed-out wait was waiting for
  // followed by done[nblocks] (unsigned, phases finished per block)
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed_int(const int *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct DepArgs {
  Geo q;
  int dim;
  double *u;
  const double *f;
  double c1, inv_c;  // h^2 / (2d), 1 / (2d)
  int rows;          // rows (2D) or planes (3D) per block
  int cols;          // 3D: y-rows per block
  int nbj;           // 3D: blocks along y (1 in 2D)
  int nblocks;
  int phases;        // 2 * sweeps
  long long max_wait_ns;
  int stall_block;   // testing: this block never publishes (-1: off)
  int cost_mode;     // S(k): COST_NONE, COST_UNIFORM or COST_LINEAR (cost.cuh)
  int kmax;
  double h2;
  DepState *st;
  unsigned *done;
};

// One colour phase on one block, in place: per interior row, the vertices of the
// phase's colour (every second one), one thread each.
__device__ void run_task(const DepArgs &a, int p, int b) {
  const Geo &q = a.q;
  const int parity = (p & 1) == 0 ? 1 : 0;  // odd vertices first
  const int64_t lo = (int64_t)(b / a.nbj) * a.rows;
  const int64_t ext = a.dim == 2 ? q.ny : q.nz;  // interior rows / planes are 1 .. ext-1
  const int64_t r0 = lo < 1 ? 1 : lo, r1 = lo + a.rows < ext ? lo + a.rows : ext;
  const int64_t ylo = (int64_t)(b % a.nbj) * a.cols;  // 3D: y-rows of the block
  const int64_t y0 = ylo < 1 ? 1 : ylo, y1 = ylo + a.cols < q.ny ? ylo + a.cols : q.ny;
  const int64_t jlo = a.dim == 2 ? r0 : y0, jhi = a.dim == 2 ? r1 : y1;
  const int64_t klo = a.dim == 2 ? 0 : r0, khi = a.dim == 2 ? 1 : r1;
  const int64_t sz = a.dim == 3 ? q.plane : 0;
  for (int64_t k = klo; k < khi; ++k)
    for (int64_t j = jlo; j < jhi; ++j) {
      // first i >= 1 with (i + j + k) & 1 == parity
      const int64_t i0 = 1 + ((parity + 1 + j + k) & 1);
      const int64_t base = k * q.plane + j * q.pitch;
      for (int64_t i = i0 + 2 * (int64_t)threadIdx.x; i < q.nx; i += 2 * D_THREADS) {
        const int64_t o = base + i;
        double s = (__ldcg(a.u + o - 1) + __ldcg(a.u + o + 1)) + (__ldcg(a.u + o - q.pitch) + __ldcg(a.u + o + q.pitch));
        if (a.dim == 3) s += __ldcg(a.u + o - sz) + __ldcg(a.u + o + sz);
        if (a.cost_mode == COST_NONE)
          a.u[o] = fma(a.c1, __ldg(a.f + o), s * a.inv_c);
        else
          a.u[o] = (a.h2 * __ldg(a.f + o) + s) / cost_diagonal(q, a.dim, a.cost_mode, a.kmax, i, j, k);
      }
    }
}

__global__ void __launch_bounds__(D_THREADS) k_depend(DepArgs a) {
  __shared__ long long task_sh;
  __shared__ int ok_sh;
  const long long ntasks = (long long)a.phases * a.nblocks;
  for (;;) {
    if (threadIdx.x == 0) {
      long long t = -1;
      if (!ld_relaxed_int(&a.st->error)) t = (long long)atomicAdd(&a.st->next_task, 1ull);
      int ok = t >= 0 && t < ntasks;
      if (ok) {
        const int p = (int)(t / a.nblocks), b = (int)(t % a.nblocks);
        if (p > 0) {
          // wait until b and its face neighbours finished phase p-1 (bounded in time)
          const unsigned long long t0 = now_ns();
          const int bk = b / a.nbj, bj = b % a.nbj, nbk = a.nblocks / a.nbj;
          for (int d = 0; d < 5 && ok; ++d) {
            const int kk = bk + (d == 1 ? -1 : d == 2 ? 1 : 0), jj = bj + (d == 3 ? -1 : d == 4 ? 1 : 0);
            if (kk < 0 || kk >= nbk || jj < 0 || jj >= a.nbj) continue;
            const int nb = kk * a.nbj + jj;
            while (ld_acquire(a.done + nb) < (unsigned)p) {
              if (ld_relaxed_int(&a.st->error) || now_ns() - t0 > (unsigned long long)a.max_wait_ns) {
                if (atomicCAS(&a.st->error, 0, 1) == 0) a.st->stalled_at = nb;
                ok = 0;
                break;
              }
              __nanosleep(100);
            }
          }
          __threadfence();
        }
      }
      task_sh = t;
      ok_sh = ok;
    }
    __syncthreads();
    const long long t = task_sh;
    const int ok = ok_sh;
    __syncthreads();  // task_sh / ok_sh are rewritten on the next round
    if (!ok) return;  // no task left, or an error: every CTA leaves
    const int p = (int)(t / a.nblocks), b = (int)(t % a.nblocks);
    run_task(a, p, b);
    __syncthreads();
    if (threadIdx.x == 0 && b != a.stall_block) {
      __threadfence();
      st_release(a.done + b, (unsigned)(p + 1));
    }
  }
}

}  // namespace

size_t depend_state_bytes(int nblocks) { return sizeof(DepState) + (size_t)nblocks * sizeof(unsigned) + 64; }

int depend_blocks(const Geo &q, int dim, int rows, int cols) {
  const int64_t ext = dim == 2 ? q.ny + 1 : q.nz + 1;
  const int64_t nbj = dim == 3 ? (q.ny + 1 + cols - 1) / cols : 1;
  return (int)((ext + rows - 1) / rows * nbj);
}

// Launches the persistent sweep; *status_host (pinned) receives the error flag and
// *stalled_host the first block whose wait timed out once the stream reaches them.
cudaError_t launch_depend_redblack(const Geo &q, int dim, double *u, const double *f, int sweeps, int rows, int cols,
                                   int ctas, long long max_wait_ns, int stall_block, void *state, int *status_host,
                                   int *stalled_host, cudaStream_t s, int cost_mode, int kmax) {
  DepArgs a{};
  a.cost_mode = cost_mode;
  a.kmax = kmax;
  a.h2 = q.h * q.h;
  a.q = q;
  a.dim = dim;
  a.u = u;
  a.f = f;
  a.c1 = q.h * q.h / (2.0 * dim);
  a.inv_c = 1.0 / (2.0 * dim);
  a.rows = rows;
  a.cols = cols;
  a.nbj = dim == 3 ? (int)((q.ny + 1 + cols - 1) / cols) : 1;
  a.nblocks = depend_blocks(q, dim, rows, cols);
  a.phases = 2 * sweeps;
  a.max_wait_ns = max_wait_ns;
  a.stall_block = stall_block;
  a.st = (DepState *)state;
  a.done = (unsigned *)((char *)state + sizeof(DepState));
  cudaError_t e = cudaMemsetAsync(state, 0, depend_state_bytes(a.nblocks), s);
  if (e) return e;
  // every CTA must be resident at once: cooperative launch of at most the occupancy
  int dev = 0, per_sm = 0, coop = 0;
  if ((e = cudaGetDevice(&dev))) return e;
  if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev))) return e;
  if (!coop) return cudaErrorNotSupported;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_depend, D_THREADS, 0))) return e;
  int grid = per_sm * device_sm_count();
  if (ctas > 0 && ctas < grid) grid = ctas;
  if (grid < 1) return cudaErrorInvalidConfiguration;
  void *args[] = {&a};
  e = cudaLaunchCooperativeKernel((const void *)k_depend, dim3(grid), dim3(D_THREADS), args, 0, s);
  if (e) return e;
  e = cudaMemcpyAsync(status_host, &a.st->error, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaMemcpyAsync(stalled_host, &a.st->stalled_at, sizeof(int), cudaMemcpyDeviceToHost, s);
  return e;
}

}  // namespace stencil
