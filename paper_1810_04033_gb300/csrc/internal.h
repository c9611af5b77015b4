// Internal declarations shared by the translation units of libstencil_gb300.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>

#include "stencil.h"

namespace stencil {

// Grid geometry as the kernels see it (element strides, not bytes).
struct Geo {
  int64_t nx, ny, nz;  // cells per axis; nz == 0 for 2D
  int64_t pitch;       // elements between x-rows
  int64_t plane;       // elements between z-planes (pitch * (ny + 1))
  double h;
};

inline Geo make_geo(const stencil_grid_t &g) {
  Geo q;
  q.nx = g.n[0];
  q.ny = g.n[1];
  q.nz = g.dim == 3 ? g.n[2] : 0;
  q.pitch = g.pitch ? g.pitch : g.n[0] + 1;
  q.plane = q.pitch * (q.ny + 1);
  q.h = g.h;
  return q;
}

// Number of elements spanned by an array of this geometry (last element + 1).
inline int64_t span_elems(const Geo &q) { return q.plane * (q.nz + 1); }

// Streaming multiprocessors of the current device (cached per device; 152 on GB300).
int device_sm_count();

// Per-device "done" flags for set-up that CUDA keeps per device, such as a kernel's
// dynamic shared-memory limit: a process may drive several GPUs and call the library
// from several host threads (the request server runs its own).
struct PerDeviceOnce {
  static constexpr int kMaxDevices = 64;
  std::atomic<bool> done[kMaxDevices];
  std::mutex mu;
};

// Raises `kernel`'s dynamic shared-memory limit to `bytes` on the current device, once
// per device; later calls on that device return at once.  Thread-safe.
template <typename Kernel>
cudaError_t set_smem_limit_once(PerDeviceOnce &once, Kernel kernel, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= PerDeviceOnce::kMaxDevices)
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (once.done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  std::lock_guard<std::mutex> lk(once.mu);
  if (once.done[dev].load(std::memory_order_relaxed)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) once.done[dev].store(true, std::memory_order_release);
  return e;
}

// Planes (or centre planes) per CTA for kernels that tile x-y and stream through z in
// chunks: the largest chunk up to cz_max that still gives about two waves of
// `ctas_per_sm` CTAs on every SM, but not below cz_min (each chunk restages its
// first neighbour plane).  Small grids thus get short chunks and more CTAs.
inline int z_chunk(int64_t tiles_xy, int64_t units, int cz_max, int cz_min, int ctas_per_sm) {
  const int64_t target = 2ll * device_sm_count() * ctas_per_sm;
  int64_t cz = (units * tiles_xy + target - 1) / target;
  if (cz > cz_max) cz = cz_max;
  if (cz < cz_min) cz = cz_min;
  return (int)cz;
}

// Launch shapes chosen by stencil_autotune or stencil_tuning_set (tuning.cu), keyed by
// the call, the grid's shape and pitch and the device's name.  chunk: 3D planes per CTA
// (or per warp) of the plane-streaming kernels, 2D rows per warp; depth: sweeps per
// pass over memory of the 2D multi-sweep smoothers (1 or 2).  0 = the built-in rule.
// Only F64 Q1 calls are tuned.  The smoothers' results do not depend on the chunk
// (exact fixed-point sums at a grid-wide scale per sweep); the 2D depth changes the
// scale (one for both sweeps of a pass) and the single-pass applies keep a per-CTA or
// per-warp scale, so those can move the rounding by units in the last place.
struct Tuning {
  int chunk = 0;
  int depth = 0;
};
Tuning tuning_lookup(int call, const Geo &q);
// The tuned chunk if one is set, clamped into [lo, hi], else `fallback`.
inline int tuned_chunk(const Tuning &t, int fallback, int lo, int hi) {
  if (t.chunk <= 0) return fallback;
  return t.chunk < lo ? lo : (t.chunk > hi ? hi : t.chunk);
}

// Flags the TMA-staged kernels set when a bounded wait on a TMA completion ran out
// (ops_fx.cu, gs_fx.cu, jac3_fx.cu, gs_lp.cu); read synchronously, optionally cleared.
cudaError_t tma_wait_flag_ops3(unsigned *value, bool clear);
cudaError_t tma_wait_flag_gs3(unsigned *value, bool clear);
cudaError_t tma_wait_flag_jac3(unsigned *value, bool clear);
cudaError_t tma_wait_flag_gs_lp(unsigned *value, bool clear);

// Error plumbing and descriptor check (api.cu).
int set_error(int code, const std::string &msg);
int check_grid(const stencil_grid_t *g);
int check_launch(const char *what);

// Library-owned scratch (api.cu), one set per (device, stream): returns a device
// pointer with at least `bytes` bytes for slot `slot`, growing with cudaMalloc when
// needed (zero-filled when allocated); nullptr on failure.  Work queued on one stream
// therefore never shares scratch with work on another stream.
enum ScratchSlot {
  SCRATCH_REDUCE = 0,
  SCRATCH_PINGPONG = 1,
  SCRATCH_BOUNDS = 2,
  SCRATCH_LP = 3,      // reduced-precision GS ping-pong
  SCRATCH_SOLVE_R = 4, // refinement: residual in the inner type
  SCRATCH_SOLVE_E = 5, // refinement: correction
  SCRATCH_NORMS = 6,   // refinement: device norms
  SCRATCH_MG = 7,      // multigrid: coarse-level arrays
  SCRATCH_DEPEND = 8,  // dependency-driven sweeps: task counter, flags, per-block progress
  SCRATCH_SLOTS = 10
};
// Pinned host scratch of the (device, stream) set.
void *host_scratch(size_t bytes, cudaStream_t stream);
void *device_scratch(int slot, size_t bytes, cudaStream_t stream);

// Residual with norms.  Reduction scratch layout (all users): an unsigned counter in
// the first 16 bytes (zero before the first call; kernels leave it zero), then the
// per-CTA partial sums.

// Fixed-point FP64 paths (gs_fx.cu): 3D coloured GS, two launches per sweep.  work
// holds 3 arrays of u's span (two int64 ping-pong buffers and 3/8 h^2 f in fixed point);
// the result always ends in u, whose boundary values are never written.
size_t gs_fx_bounds_bytes();
// Per-call pre-pass of the multi-sweep GS and Jacobi launchers: clears the bounds, takes max |u| and
// max |f| (interior), and writes GF = 3/8 h^2 f as fixed point (0 off the interior).
cudaError_t launch_gs_prepass(const Geo &q, int dim, const double *u, const double *f, long long *GF,
                              void *bounds, int sweeps, cudaStream_t s);
cudaError_t launch_gs_sweeps_fx3(const Geo &q, double *u, const double *f, int sweeps,
                                 double *work, void *bounds, cudaStream_t s);

// Fixed-point out-of-place 3D operations (ops_fx.cu).  The residual needs
// ops_fx_reduce_bytes(q) bytes of zero-initialised scratch (left zeroed).
size_t ops_fx_reduce_bytes(const Geo &q);
cudaError_t launch_apply_stencil_fx3(const Geo &q, const double *u, double *y, cudaStream_t s);
cudaError_t launch_apply_elementwise_fx3(const Geo &q, const double *u, double *y, cudaStream_t s);
cudaError_t launch_jacobi_fx3(const Geo &q, const double *u, const double *f, double *unew,
                              double omega, cudaStream_t s);
// 2D (ops2d_fx.cu)
size_t ops2_reduce_bytes(const Geo &q);
cudaError_t launch_apply_fx2(const Geo &q, const double *u, double *y, bool elementwise, cudaStream_t s);
cudaError_t launch_jacobi_fx2(const Geo &q, const double *u, const double *f, double *unew, double omega,
                              cudaStream_t s);
cudaError_t launch_residual_fx2(const Geo &q, const double *u, const double *f, double *r, double *norms2,
                                void *scratch, cudaStream_t s);
// 2D coloured GS, one launch per sweep; work and bounds as for the 3D form.
cudaError_t launch_gs_sweeps_fx2(const Geo &q, double *u, const double *f, int sweeps, double *work,
                                 void *bounds, cudaStream_t s);
// Multi-sweep damped Jacobi, 2D, 0 < omega <= 1, int64 fixed point between sweeps.
// A: one u-sized buffer; scratch: two; bounds: gs_fx_bounds_bytes().  Result in u.
cudaError_t launch_jacobi_sweeps_fx2(const Geo &q, double *u, const double *f, int sweeps, double omega, double *A,
                                     double *scratch, void *bounds, cudaStream_t s);
cudaError_t launch_jacobi_sweeps_fx3(const Geo &q, double *u, const double *f, int sweeps, double omega, double *A,
                                     double *scratch, void *bounds, cudaStream_t s);
// out_kind: r stored as 0 = FP64, 1 = FP32, 2 = bf16 (r is an element pointer of that
// type passed as double*; the layout is u's).
cudaError_t launch_residual_fx3(const Geo &q, const double *u, const double *f, double *r,
                                double *norms2, void *scratch, cudaStream_t s, int out_kind = 0);

// Reduced-precision coloured GS, 3D (gs_lp.cu): work has u's span of the same type.
cudaError_t launch_gs_sweeps_f32_3d(const Geo &q, float *u, const float *f, int sweeps, float *work,
                                    cudaStream_t s);
cudaError_t launch_gs_sweeps_bf16_3d(const Geo &q, void *u, const void *f, int sweeps, void *work,
                                     cudaStream_t s);

// x += e on interior vertices, e of element type dtype (solve.cu).
cudaError_t launch_add_correction(const Geo &q, int dim, double *x, const void *e, int dtype, cudaStream_t s);

// 5/7-point finite differences with red-black GS (fd.cu); F64, 2D and 3D.
size_t fd_reduce_bytes(const Geo &q);
cudaError_t launch_fd_apply(const Geo &q, int dim, const double *u, double *y, cudaStream_t s);
cudaError_t launch_fd_jacobi(const Geo &q, int dim, const double *u, const double *f, double *unew, double omega,
                             cudaStream_t s);
cudaError_t launch_fd_residual(const Geo &q, int dim, const double *u, const double *f, double *r, double *norms2,
                               void *scratch, cudaStream_t s);
cudaError_t launch_fd_gs_redblack(const Geo &q, int dim, double *u, const double *f, int sweeps, cudaStream_t s);

// Dependency-driven red-black sweeps (depend.cu), op FD, F64.
size_t depend_state_bytes(int nblocks);
int depend_blocks(const Geo &q, int dim, int rows, int cols);
cudaError_t launch_depend_redblack(const Geo &q, int dim, double *u, const double *f, int sweeps, int rows, int cols,
                                   int ctas, long long max_wait_ns, int stall_block, void *state, int *status_host,
                                   int *stalled_host, cudaStream_t s, int cost_mode = 0, int kmax = 0);
// Red-black sweeps with expensive stencil evaluations S(k) (fd.cu, cost.cuh).
cudaError_t launch_fd_gs_redblack_cost(const Geo &q, int dim, double *u, const double *f, int sweeps, int mode,
                                       int kmax, cudaStream_t s);

// Geometric multigrid (mg.cu).  Coarse grids are dense (pitch n_c + 1): n/2 per axis
// when all n are even, ceil(n/2) when all n are equal; none (false) below n = 4.
bool mg_coarse(const Geo &qf, int dim, Geo &qc);
int mg_levels(const Geo &q, int dim, int max_levels);
size_t mg_work_bytes(const Geo &q0, int dim, int levels);    // coarse-level arrays
size_t mg_reduce_bytes(const Geo &q0, int dim, int levels);  // residual reduction scratch
cudaError_t launch_mg_restrict(const Geo &qf, const Geo &qc, int dim, const double *rf, double *rc, cudaStream_t s);
cudaError_t launch_mg_prolong_add(const Geo &qf, const Geo &qc, int dim, const double *ec, double *uf,
                                  cudaStream_t s);

// One V-cycle, stream-ordered.  setup() carves the coarse-level arrays out of `work`
// (mg_work_bytes); gs_work / gs_bounds are the multi-sweep GS workspace of the finest
// grid (reused on every level), norms 2 doubles and red the residual reduction scratch
// (mg_reduce_bytes), both device.
class MgCycle {
 public:
  static constexpr int kMaxLevels = 40;
  bool setup(const Geo &q0, int dim, int levels, int pre, int post, int coarse_sweeps, void *work,
             double *gs_work, void *gs_bounds, double *norms, void *red, cudaStream_t s);
  cudaError_t run(double *u0, const double *f0);

 private:
  cudaError_t level(int l, double *u, const double *f);
  cudaError_t smooth(const Geo &q, double *u, const double *f, int sweeps);
  Geo q_[kMaxLevels];
  double *u_[kMaxLevels], *f_[kMaxLevels], *r_[kMaxLevels];
  int dim_ = 3, levels_ = 1, pre_ = 2, post_ = 2, coarse_sweeps_ = 20;
  double *gs_work_ = nullptr;
  void *gs_bounds_ = nullptr;
  double *norms_ = nullptr;
  void *red_ = nullptr;
  cudaStream_t s_ = nullptr;
};

}  // namespace stencil
