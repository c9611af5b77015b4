// C ABI entry points of libstencil_gb300: argument checks, scratch management and
// dispatch to the kernels.  See include/stencil.h for the contract of each call.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cudaTypedefs.h>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "tma.cuh"

namespace stencil {

static thread_local std::string g_last_error;

int set_error(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

int check_launch(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return set_error(STENCIL_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return STENCIL_OK;
}

int device_sm_count() {
  // host threads may race to fill an entry; they all store the same value
  static std::atomic<int> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int n = cached[dev].load(std::memory_order_relaxed);
  if (!n) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    cached[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

// ------------------------------------------------------------ TMA tensor maps
bool tma_plane_map(const Geo &q, const void *base, int box_w, int box_h, CUtensorMap *map) {
  return tma_plane_map_elem(q, base, 8, box_w, box_h, map);
}

bool tma_plane_map_elem(const Geo &q, const void *base, int elem_bytes, int box_w, int box_h, CUtensorMap *map) {
  // strides and base need 16-byte alignment
  if ((uintptr_t)base % 16 || (q.pitch * elem_bytes) % 16) return false;
  if (elem_bytes != 8 && elem_bytes != 4 && elem_bytes != 2) return false;
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  std::call_once(once, [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) ==
            cudaSuccess &&
        qr == cudaDriverEntryPointSuccess)
      encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  });
  if (!encode) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)q.nx + 1, (cuuint64_t)q.ny + 1, (cuuint64_t)q.nz + 1};
  const cuuint64_t strides[2] = {(cuuint64_t)q.pitch * elem_bytes, (cuuint64_t)q.plane * elem_bytes};
  const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUtensorMapDataType dt = elem_bytes == 8   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                 : elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                   : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  return encode(map, dt, 3, const_cast<void *>(base), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ------------------------------------------------------------ per-stream scratch
namespace {
constexpr int kMaxDevices = 64;
struct Scratch {
  int device;
  cudaStream_t stream;
  void *ptr[SCRATCH_SLOTS];
  size_t bytes[SCRATCH_SLOTS];
  void *host;
  size_t host_bytes;
};
std::mutex g_scratch_mu;
std::vector<Scratch> g_scratch;
}  // namespace

void *device_scratch(int slot, size_t bytes, cudaStream_t stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  Scratch *s = nullptr;
  for (auto &e : g_scratch)
    if (e.device == dev && e.stream == stream) s = &e;
  if (!s) {
    g_scratch.push_back(Scratch{dev, stream, {nullptr}, {0}, nullptr, 0});
    s = &g_scratch.back();
  }
  if (s->bytes[slot] >= bytes && s->ptr[slot]) return s->ptr[slot];
  if (s->ptr[slot]) {
    // the old buffer may still be in use by work queued on this stream
    cudaStreamSynchronize(stream);
    cudaFree(s->ptr[slot]);
    s->ptr[slot] = nullptr;
    s->bytes[slot] = 0;
  }
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  // reduction counters must start at zero
  if (cudaMemset(p, 0, bytes) != cudaSuccess) {
    cudaFree(p);
    return nullptr;
  }
  s->ptr[slot] = p;
  s->bytes[slot] = bytes;
  return p;
}

void *host_scratch(size_t bytes, cudaStream_t stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  // make sure the set exists
  if (!device_scratch(SCRATCH_NORMS, 64, stream)) return nullptr;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  for (auto &e : g_scratch) {
    if (e.device != dev || e.stream != stream) continue;
    if (e.host && e.host_bytes >= bytes) return e.host;
    if (e.host) {
      cudaStreamSynchronize(stream);
      cudaFreeHost(e.host);
      e.host = nullptr;
    }
    if (cudaMallocHost(&e.host, bytes) != cudaSuccess) {
      cudaGetLastError();
      e.host = nullptr;
      return nullptr;
    }
    e.host_bytes = bytes;
    return e.host;
  }
  return nullptr;
}

static int release_scratch() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return set_error(STENCIL_ECUDA, "cudaGetDevice failed");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  cudaDeviceSynchronize();
  for (auto it = g_scratch.begin(); it != g_scratch.end();) {
    if (it->device == dev) {
      for (int i = 0; i < SCRATCH_SLOTS; ++i)
        if (it->ptr[i]) cudaFree(it->ptr[i]);
      if (it->host) cudaFreeHost(it->host);
      it = g_scratch.erase(it);
    } else {
      ++it;
    }
  }
  return STENCIL_OK;
}

// ------------------------------------------------------------ argument checks
static size_t elem_size(int dtype) {
  switch (dtype) {
    case STENCIL_F64: return 8;
    case STENCIL_F32: return 4;
    case STENCIL_BF16: return 2;
    default: return 0;
  }
}

// Entry points that implement the Q1 operator only.
static int require_q1(const stencil_grid_t *g, const char *what) {
  if (g->op != STENCIL_OP_Q1)
    return set_error(STENCIL_EINVAL, std::string(what) + ": the Q1 operator only (op = STENCIL_OP_Q1)");
  return STENCIL_OK;
}

int check_grid(const stencil_grid_t *g) {
  if (!g) return set_error(STENCIL_EINVAL, "grid descriptor is NULL");
  if (g->dim != 2 && g->dim != 3) return set_error(STENCIL_EINVAL, "dim must be 2 or 3");
  if (!elem_size(g->dtype)) return set_error(STENCIL_EINVAL, "unknown dtype");
  if (g->op != STENCIL_OP_Q1 && g->op != STENCIL_OP_FD) return set_error(STENCIL_EINVAL, "unknown operator");
  if (g->op == STENCIL_OP_FD && g->dtype != STENCIL_F64)
    return set_error(STENCIL_EINVAL, "the finite-difference operator supports F64 only");
  const int64_t lim = (int64_t)1 << 31;
  for (int a = 0; a < g->dim; ++a)
    if (g->n[a] < 1 || g->n[a] >= lim)
      return set_error(STENCIL_EINVAL, "cells per axis must be in [1, 2^31)");
  const int64_t pitch = g->pitch ? g->pitch : g->n[0] + 1;
  if (pitch < g->n[0] + 1) return set_error(STENCIL_EINVAL, "pitch < n[0] + 1");
  if (!(g->h > 0.0) || !std::isfinite(g->h))
    return set_error(STENCIL_EINVAL, "h must be finite and > 0");
  // total span must fit comfortably in int64 element offsets
  const double span = (double)pitch * (double)(g->n[1] + 1) *
                      (double)(g->dim == 3 ? g->n[2] + 1 : 1);
  if (span > 9.0e15) return set_error(STENCIL_EINVAL, "array too large");
  return STENCIL_OK;
}

static int check_ptr(const void *p, const stencil_grid_t *g, const char *name) {
  if (!p) return set_error(STENCIL_EINVAL, std::string(name) + " is NULL");
  if ((uintptr_t)p % elem_size(g->dtype))
    return set_error(STENCIL_EINVAL, std::string(name) + " is not aligned to its element size");
  return STENCIL_OK;
}

static bool overlap(const void *a, const void *b, size_t bytes) {
  const char *x = (const char *)a, *y = (const char *)b;
  return x < y + bytes && y < x + bytes;
}

// [a, a + na) and [b, b + nb) intersect.
static bool overlap2(const void *a, size_t na, const void *b, size_t nb) {
  const char *x = (const char *)a, *y = (const char *)b;
  return x < y + nb && y < x + na;
}

// ------------------------------------------------------------ call workspaces
// The device workspace of a call is at most two parts, each starting on a 256-byte
// boundary of one buffer.  A caller that passes its own buffer (at least total() bytes,
// 256-byte aligned) gets no allocation from the call; a NULL buffer selects the
// library's per-(device, stream) scratch slots.
static size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

struct WsNeed {
  size_t part[2] = {0, 0};
  int slot[2] = {0, 0};
  bool zero_head = false;  // part 0 starts with a reduction counter that must be 0
  size_t total() const { return part[1] ? round256(part[0]) + part[1] : part[0]; }
};

static WsNeed smooth_coloured_need(const stencil_grid_t *g, int sweeps) {
  WsNeed w;
  if (sweeps <= 0 || g->op == STENCIL_OP_FD) return w;
  const size_t span = (size_t)span_elems(make_geo(*g));
  if (g->dtype != STENCIL_F64) {
    w.part[0] = span * elem_size(g->dtype);
    w.slot[0] = SCRATCH_LP;
    return w;
  }
  w.part[0] = 3 * span * 8;  // two int64 ping-pong copies and 3/8 h^2 f in fixed point
  w.slot[0] = SCRATCH_PINGPONG;
  w.part[1] = gs_fx_bounds_bytes();
  w.slot[1] = SCRATCH_BOUNDS;
  return w;
}

// Multi-sweep Q1 Jacobi runs its fast path for 0 < omega <= 1; the size does not
// depend on omega (other omegas need less).
static WsNeed smooth_jacobi_need(const stencil_grid_t *g, int sweeps) {
  WsNeed w;
  if (g->op != STENCIL_OP_Q1 || sweeps < 2) return w;
  w.part[0] = 2 * (size_t)span_elems(make_geo(*g)) * 8;
  w.slot[0] = SCRATCH_PINGPONG;
  w.part[1] = gs_fx_bounds_bytes();
  w.slot[1] = SCRATCH_BOUNDS;
  return w;
}

static WsNeed residual_need(const stencil_grid_t *g) {
  WsNeed w;
  const Geo q = make_geo(*g);
  w.part[0] = g->op == STENCIL_OP_FD ? fd_reduce_bytes(q) : g->dim == 3 ? ops_fx_reduce_bytes(q) : ops2_reduce_bytes(q);
  w.slot[0] = SCRATCH_REDUCE;
  w.zero_head = true;
  return w;
}

// Checks a caller workspace against the need (synchronously, before any device work).
static int check_ws(const WsNeed &need, const void *ws, size_t ws_bytes, const char *what) {
  if (!ws) return STENCIL_OK;
  if ((uintptr_t)ws % 256)
    return set_error(STENCIL_EINVAL, std::string(what) + ": workspace must be 256-byte aligned");
  if (ws_bytes < need.total())
    return set_error(STENCIL_EINVAL, std::string(what) + ": workspace too small (" + std::to_string(ws_bytes) +
                                         " bytes given, " + std::to_string(need.total()) + " needed)");
  return STENCIL_OK;
}

// Resolves the parts: carved from the caller's buffer, or the library's scratch.
static int take_ws(const WsNeed &need, void *ws, cudaStream_t s, void *out[2], const char *what) {
  out[0] = out[1] = nullptr;
  if (ws) {
    out[0] = need.part[0] ? ws : nullptr;
    out[1] = need.part[1] ? (char *)ws + round256(need.part[0]) : nullptr;
    if (need.zero_head && cudaMemsetAsync(ws, 0, 16, s) != cudaSuccess)
      return set_error(STENCIL_ECUDA, std::string(what) + ": clearing the workspace counter failed");
    return STENCIL_OK;
  }
  for (int i = 0; i < 2; ++i)
    if (need.part[i] && !(out[i] = device_scratch(need.slot[i], need.part[i], s)))
      return set_error(STENCIL_ENOMEM, std::string(what) + ": workspace allocation failed");
  return STENCIL_OK;
}

}  // namespace stencil

using namespace stencil;

extern "C" {

int stencil_version(void) { return 10000; }

const char *stencil_last_error(void) { return g_last_error.c_str(); }

int stencil_release_workspace(void) { return release_scratch(); }

int stencil_device_status(uint32_t *flags, int clear) {
  if (!flags) return set_error(STENCIL_EINVAL, "device_status: flags is NULL");
  *flags = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return set_error(STENCIL_ECUDA, std::string("device_status: ") + cudaGetErrorString(e));
  cudaError_t (*const readers[4])(unsigned *, bool) = {tma_wait_flag_ops3, tma_wait_flag_gs3, tma_wait_flag_jac3,
                                                       tma_wait_flag_gs_lp};
  for (int i = 0; i < 4; ++i) {
    unsigned v = 0;
    e = readers[i](&v, clear != 0);
    if (e != cudaSuccess) return set_error(STENCIL_ECUDA, std::string("device_status: ") + cudaGetErrorString(e));
    if (v) *flags |= 1u << i;
  }
  return STENCIL_OK;
}

int stencil_workspace_size(const stencil_grid_t *g, int call, int sweeps, size_t *bytes) {
  if (!bytes) return set_error(STENCIL_EINVAL, "workspace_size: bytes is NULL");
  *bytes = 0;
  int rc = check_grid(g);
  if (rc) return rc;
  if (sweeps < 0) return set_error(STENCIL_EINVAL, "workspace_size: sweeps < 0");
  switch (call) {
    case STENCIL_CALL_SMOOTH_COLOURED: *bytes = smooth_coloured_need(g, sweeps).total(); break;
    case STENCIL_CALL_SMOOTH_JACOBI: *bytes = smooth_jacobi_need(g, sweeps).total(); break;
    case STENCIL_CALL_RESIDUAL: *bytes = residual_need(g).total(); break;
    case STENCIL_CALL_APPLY_ELEMENTWISE:
    case STENCIL_CALL_APPLY_STENCIL: break;
    default: return set_error(STENCIL_EINVAL, "workspace_size: unknown call");
  }
  return STENCIL_OK;
}

int stencil_apply(const stencil_grid_t *g, const void *u, void *y, int form, void *stream) {
  int rc = check_grid(g);
  if (rc) return rc;
  if ((rc = check_ptr(u, g, "u")) || (rc = check_ptr(y, g, "y"))) return rc;
  if (form != STENCIL_FORM_ELEMENTWISE && form != STENCIL_FORM_STENCIL)
    return set_error(STENCIL_EINVAL, "unknown apply form");
  if (g->dtype != STENCIL_F64) return set_error(STENCIL_EINVAL, "apply supports F64 only");
  const Geo q = make_geo(*g);
  if (overlap(u, y, (size_t)span_elems(q) * 8))
    return set_error(STENCIL_EINVAL, "u and y overlap");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (g->op == STENCIL_OP_FD) {
    if (form != STENCIL_FORM_STENCIL)
      return set_error(STENCIL_EINVAL, "apply: the finite-difference operator has the stencil form only");
    e = launch_fd_apply(q, g->dim, (const double *)u, (double *)y, s);
  } else if (g->dim == 2)
    e = launch_apply_fx2(q, (const double *)u, (double *)y, form == STENCIL_FORM_ELEMENTWISE, s);
  else if (form == STENCIL_FORM_STENCIL)
    e = launch_apply_stencil_fx3(q, (const double *)u, (double *)y, s);
  else
    e = launch_apply_elementwise_fx3(q, (const double *)u, (double *)y, s);
  if (e != cudaSuccess) return set_error(STENCIL_ECUDA, std::string("apply: ") + cudaGetErrorString(e));
  return STENCIL_OK;
}

int stencil_smooth_coloured(const stencil_grid_t *g, void *u, const void *f, int sweeps, void *ws,
                            size_t ws_bytes, void *stream) {
  int rc = check_grid(g);
  if (rc) return rc;
  if ((rc = check_ptr(u, g, "u")) || (rc = check_ptr(f, g, "f"))) return rc;
  if (sweeps < 0) return set_error(STENCIL_EINVAL, "sweeps < 0");
  if (g->dtype != STENCIL_F64 && g->dim != 3)
    return set_error(STENCIL_EINVAL, "smooth_coloured: F32/BF16 storage is 3D only");
  const Geo q = make_geo(*g);
  const size_t esz = elem_size(g->dtype);
  if (overlap(u, f, (size_t)span_elems(q) * esz)) return set_error(STENCIL_EINVAL, "u and f overlap");
  const WsNeed need = smooth_coloured_need(g, sweeps);
  if ((rc = check_ws(need, ws, ws_bytes, "smooth_coloured"))) return rc;
  const size_t wsb = need.total(), ub = (size_t)span_elems(q) * esz;
  if (ws && wsb && (overlap2(ws, wsb, u, ub) || overlap2(ws, wsb, f, ub)))
    return set_error(STENCIL_EINVAL, "smooth_coloured: workspace overlaps u or f");
  if (sweeps == 0) return STENCIL_OK;
  cudaStream_t s = (cudaStream_t)stream;
  void *part[2];
  if ((rc = take_ws(need, ws, s, part, "smooth_coloured"))) return rc;
  cudaError_t e;
  if (g->op == STENCIL_OP_FD) {
    e = launch_fd_gs_redblack(q, g->dim, (double *)u, (const double *)f, sweeps, s);
  } else if (g->dtype != STENCIL_F64) {
    e = g->dtype == STENCIL_F32
            ? launch_gs_sweeps_f32_3d(q, (float *)u, (const float *)f, sweeps, (float *)part[0], s)
            : launch_gs_sweeps_bf16_3d(q, u, f, sweeps, part[0], s);
  } else if (g->dim == 3) {
    e = launch_gs_sweeps_fx3(q, (double *)u, (const double *)f, sweeps, (double *)part[0], part[1], s);
  } else {
    e = launch_gs_sweeps_fx2(q, (double *)u, (const double *)f, sweeps, (double *)part[0], part[1], s);
  }
  if (e != cudaSuccess)
    return set_error(STENCIL_ECUDA, std::string("smooth_coloured: ") + cudaGetErrorString(e));
  return STENCIL_OK;
}

int stencil_smooth_jacobi(const stencil_grid_t *g, void *u, const void *f, void *work,
                          int sweeps, double omega, void *ws, size_t ws_bytes, void *stream) {
  int rc = check_grid(g);
  if (rc) return rc;
  if ((rc = check_ptr(u, g, "u")) || (rc = check_ptr(f, g, "f")) ||
      (rc = check_ptr(work, g, "work")))
    return rc;
  if (sweeps < 0) return set_error(STENCIL_EINVAL, "sweeps < 0");
  if (!std::isfinite(omega)) return set_error(STENCIL_EINVAL, "omega must be finite");
  if (g->dtype != STENCIL_F64) return set_error(STENCIL_EINVAL, "jacobi supports F64 only");
  const Geo q = make_geo(*g);
  const size_t bytes = (size_t)span_elems(q) * 8;
  if (overlap(u, f, bytes) || overlap(u, work, bytes) || overlap(f, work, bytes))
    return set_error(STENCIL_EINVAL, "u, f and work must not overlap");
  const WsNeed need = smooth_jacobi_need(g, sweeps);
  if ((rc = check_ws(need, ws, ws_bytes, "smooth_jacobi"))) return rc;
  const size_t wsb = need.total();
  if (ws && wsb && (overlap2(ws, wsb, u, bytes) || overlap2(ws, wsb, f, bytes) || overlap2(ws, wsb, work, bytes)))
    return set_error(STENCIL_EINVAL, "smooth_jacobi: workspace overlaps u, f or work");
  cudaStream_t s = (cudaStream_t)stream;
  if (g->op == STENCIL_OP_Q1 && sweeps >= 2 && omega > 0.0 && omega <= 1.0) {
    void *part[2];
    if ((rc = take_ws(need, ws, s, part, "smooth_jacobi"))) return rc;
    void *scr = part[0], *bnd = part[1];
    cudaError_t e =
        g->dim == 2 ? launch_jacobi_sweeps_fx2(q, (double *)u, (const double *)f, sweeps, omega, (double *)work,
                                               (double *)scr, bnd, s)
                    : launch_jacobi_sweeps_fx3(q, (double *)u, (const double *)f, sweeps, omega, (double *)work,
                                               (double *)scr, bnd, s);
    if (e != cudaSuccess) return set_error(STENCIL_ECUDA, std::string("jacobi: ") + cudaGetErrorString(e));
    return STENCIL_OK;
  }
  double *a = (double *)u, *b = (double *)work;
  for (int it = 0; it < sweeps; ++it) {
    cudaError_t e = g->op == STENCIL_OP_FD ? launch_fd_jacobi(q, g->dim, a, (const double *)f, b, omega, s)
                    : g->dim == 3         ? launch_jacobi_fx3(q, a, (const double *)f, b, omega, s)
                                          : launch_jacobi_fx2(q, a, (const double *)f, b, omega, s);
    if (e != cudaSuccess) return set_error(STENCIL_ECUDA, std::string("jacobi: ") + cudaGetErrorString(e));
    double *t = a;
    a = b;
    b = t;
  }
  if (a != (double *)u) {
    cudaError_t e = cudaMemcpyAsync(u, a, bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return set_error(STENCIL_ECUDA, std::string("jacobi copy: ") + cudaGetErrorString(e));
  }
  return STENCIL_OK;
}

int stencil_jacobi_step(const stencil_grid_t *g, const void *u_in, const void *f, void *u_out,
                        double omega, void *stream) {
  int rc = check_grid(g);
  if (rc) return rc;
  if ((rc = check_ptr(u_in, g, "u_in")) || (rc = check_ptr(f, g, "f")) ||
      (rc = check_ptr(u_out, g, "u_out")))
    return rc;
  if (!std::isfinite(omega)) return set_error(STENCIL_EINVAL, "omega must be finite");
  if (g->dtype != STENCIL_F64) return set_error(STENCIL_EINVAL, "jacobi supports F64 only");
  const Geo q = make_geo(*g);
  const size_t bytes = (size_t)span_elems(q) * 8;
  if (overlap(u_out, u_in, bytes) || overlap(u_out, f, bytes))
    return set_error(STENCIL_EINVAL, "u_out overlaps an input");
  cudaError_t e =
      g->op == STENCIL_OP_FD
          ? launch_fd_jacobi(q, g->dim, (const double *)u_in, (const double *)f, (double *)u_out, omega,
                             (cudaStream_t)stream)
      : g->dim == 3 ? launch_jacobi_fx3(q, (const double *)u_in, (const double *)f, (double *)u_out, omega,
                                      (cudaStream_t)stream)
                  : launch_jacobi_fx2(q, (const double *)u_in, (const double *)f, (double *)u_out, omega,
                                      (cudaStream_t)stream);
  if (e != cudaSuccess) return set_error(STENCIL_ECUDA, std::string("jacobi: ") + cudaGetErrorString(e));
  return STENCIL_OK;
}

int stencil_residual(const stencil_grid_t *g, const void *u, const void *f, void *r,
                     double *d_norms2, void *ws, size_t ws_bytes, void *stream) {
  int rc = check_grid(g);
  if (rc) return rc;
  if ((rc = check_ptr(u, g, "u")) || (rc = check_ptr(f, g, "f"))) return rc;
  if (r && (rc = check_ptr(r, g, "r"))) return rc;
  if (!d_norms2 || (uintptr_t)d_norms2 % 8) return set_error(STENCIL_EINVAL, "d_norms2 NULL or misaligned");
  if (g->dtype != STENCIL_F64) return set_error(STENCIL_EINVAL, "residual supports F64 only");
  const Geo q = make_geo(*g);
  const size_t bytes = (size_t)span_elems(q) * 8;
  if (r && (overlap(r, u, bytes) || overlap(r, f, bytes)))
    return set_error(STENCIL_EINVAL, "r overlaps u or f");
  const WsNeed need = residual_need(g);
  if ((rc = check_ws(need, ws, ws_bytes, "residual"))) return rc;
  const size_t wsb = need.total();
  if (ws && (overlap2(ws, wsb, u, bytes) || overlap2(ws, wsb, f, bytes) || (r && overlap2(ws, wsb, r, bytes)) ||
             overlap2(ws, wsb, d_norms2, 16)))
    return set_error(STENCIL_EINVAL, "residual: workspace overlaps an argument");
  void *part[2];
  if ((rc = take_ws(need, ws, (cudaStream_t)stream, part, "residual"))) return rc;
  void *scratch = part[0];
  cudaError_t e =
      g->op == STENCIL_OP_FD
          ? launch_fd_residual(q, g->dim, (const double *)u, (const double *)f, (double *)r, d_norms2, scratch,
                               (cudaStream_t)stream)
      : g->dim == 3 ? launch_residual_fx3(q, (const double *)u, (const double *)f, (double *)r, d_norms2,
                                        scratch, (cudaStream_t)stream)
                  : launch_residual_fx2(q, (const double *)u, (const double *)f, (double *)r, d_norms2,
                                        scratch, (cudaStream_t)stream);
  if (e != cudaSuccess) return set_error(STENCIL_ECUDA, std::string("residual: ") + cudaGetErrorString(e));
  return STENCIL_OK;
}

int stencil_solve(const stencil_grid_t *g, double *u, const double *f, const stencil_solve_opts_t *opts,
                  stencil_solve_info_t *info, void *stream) {
  int rc = check_grid(g);
  if (rc) return rc;
  if (g->dtype != STENCIL_F64) return set_error(STENCIL_EINVAL, "solve: u and f must be F64");
  if ((rc = require_q1(g, "solve"))) return rc;
  if ((rc = check_ptr(u, g, "u")) || (rc = check_ptr(f, g, "f"))) return rc;
  if (!opts) return set_error(STENCIL_EINVAL, "solve: opts is NULL");
  if (!(opts->rel_tol >= 0.0) || opts->max_outer < 0 || opts->inner_sweeps < 1)
    return set_error(STENCIL_EINVAL, "solve: need rel_tol >= 0, max_outer >= 0, inner_sweeps >= 1");
  const int inner = opts->inner_dtype;
  if (inner != STENCIL_F64 && inner != STENCIL_F32 && inner != STENCIL_BF16)
    return set_error(STENCIL_EINVAL, "solve: unknown inner_dtype");
  if (inner != STENCIL_F64 && g->dim != 3)
    return set_error(STENCIL_EINVAL, "solve: FP32/BF16 inner sweeps are 3D only");
  const Geo q = make_geo(*g);
  const size_t span = (size_t)span_elems(q);
  if (overlap(u, f, span * 8)) return set_error(STENCIL_EINVAL, "u and f overlap");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t esz = elem_size(inner);
  void *r = device_scratch(SCRATCH_SOLVE_R, span * esz, s);
  void *e = device_scratch(SCRATCH_SOLVE_E, span * esz, s);
  double *dn = (double *)device_scratch(SCRATCH_NORMS, 64, s);
  const size_t red = g->dim == 3 ? ops_fx_reduce_bytes(q) : ops2_reduce_bytes(q);
  void *red_scr = device_scratch(SCRATCH_REDUCE, red, s);
  double *hn = (double *)host_scratch(64, s);
  void *work = nullptr;
  if (inner == STENCIL_F64)
    work = device_scratch(SCRATCH_PINGPONG, 3 * span * 8, s);
  else
    work = device_scratch(SCRATCH_LP, span * esz, s);
  void *bnd = device_scratch(SCRATCH_BOUNDS, gs_fx_bounds_bytes(), s);
  if (!r || !e || !dn || !red_scr || !hn || !work || !bnd)
    return set_error(STENCIL_ENOMEM, "solve: workspace allocation failed");
  const int out_kind = inner == STENCIL_F64 ? 0 : (inner == STENCIL_F32 ? 1 : 2);
  int k = 0;
  double rho = 0.0;
  bool conv = false;
  for (;;) {
    cudaError_t ce = g->dim == 3
                         ? launch_residual_fx3(q, u, f, (double *)r, dn, red_scr, s, out_kind)
                         : launch_residual_fx2(q, u, f, (double *)r, dn, red_scr, s);
    if (!ce) ce = cudaMemcpyAsync(hn, dn, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (!ce) ce = cudaStreamSynchronize(s);
    if (ce) return set_error(STENCIL_ECUDA, std::string("solve: ") + cudaGetErrorString(ce));
    rho = hn[1] > 0.0 ? std::sqrt(hn[0]) / std::sqrt(hn[1]) : std::sqrt(hn[0]);
    if (info && info->relres_history) info->relres_history[k] = rho;
    if (rho <= opts->rel_tol) {
      conv = true;
      break;
    }
    if (k >= opts->max_outer) break;
    ce = cudaMemsetAsync(e, 0, span * esz, s);
    if (!ce) {
      if (inner == STENCIL_F64)
        ce = g->dim == 3 ? launch_gs_sweeps_fx3(q, (double *)e, (const double *)r, opts->inner_sweeps,
                                                (double *)work, bnd, s)
                         : launch_gs_sweeps_fx2(q, (double *)e, (const double *)r, opts->inner_sweeps,
                                                (double *)work, bnd, s);
      else if (inner == STENCIL_F32)
        ce = launch_gs_sweeps_f32_3d(q, (float *)e, (const float *)r, opts->inner_sweeps, (float *)work, s);
      else
        ce = launch_gs_sweeps_bf16_3d(q, e, r, opts->inner_sweeps, work, s);
    }
    if (!ce) ce = launch_add_correction(q, g->dim, u, e, inner, s);
    if (ce) return set_error(STENCIL_ECUDA, std::string("solve: ") + cudaGetErrorString(ce));
    ++k;
  }
  if (info) {
    info->iterations = k;
    info->converged = conv ? 1 : 0;
    info->relres = rho;
  }
  if (!conv) return set_error(STENCIL_ENOTCONV, "solve: max_outer reached before rel_tol");
  return STENCIL_OK;
}

// ------------------------------------------------------------ dependency-driven sweeps

static int smooth_depend_impl(const stencil_grid_t *g, double *u, const double *f, int sweeps,
                              stencil_depend_opts_t *opts, int cost_mode, int kmax, void *stream) {
  if (!opts) return set_error(STENCIL_EINVAL, "smooth_depend: opts is NULL");
  if (sweeps < 0 || opts->rows < 0 || opts->cols < 0 || opts->ctas < 0 || opts->max_wait_ns < 0 ||
      opts->test_stall < 0)
    return set_error(STENCIL_EINVAL, "smooth_depend: negative argument");
  const Geo q = make_geo(*g);
  opts->stalled_at = -1;
  if (sweeps == 0) return STENCIL_OK;
  const int rows = opts->rows > 0 ? opts->rows : (g->dim == 2 ? 8 : 1);
  const int cols = opts->cols > 0 ? opts->cols : 32;
  const int nb = depend_blocks(q, g->dim, rows, cols);
  cudaStream_t s = (cudaStream_t)stream;
  void *state = device_scratch(SCRATCH_DEPEND, depend_state_bytes(nb), s);
  int *hs = (int *)host_scratch(64, s);
  if (!state || !hs) return set_error(STENCIL_ENOMEM, "smooth_depend: workspace allocation failed");
  const long long wait = opts->max_wait_ns > 0 ? opts->max_wait_ns : 1000000000ll;
  cudaError_t e = launch_depend_redblack(q, g->dim, u, f, sweeps, rows, cols, opts->ctas, wait, opts->test_stall - 1,
                                         state, hs, hs + 1, s, cost_mode, kmax);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return set_error(STENCIL_ECUDA, std::string("smooth_depend: ") + cudaGetErrorString(e));
  if (hs[0]) {
    opts->stalled_at = hs[1];
    return set_error(STENCIL_ETIMEDOUT, "smooth_depend: a dependency wait exceeded max_wait_ns (block " +
                                            std::to_string(hs[1]) + ")");
  }
  return STENCIL_OK;
}

static int check_fd_uf(const stencil_grid_t *g, const double *u, const double *f, const char *what) {
  int rc = check_grid(g);
  if (rc) return rc;
  if (g->op != STENCIL_OP_FD) return set_error(STENCIL_EINVAL, std::string(what) + ": needs op = STENCIL_OP_FD");
  if ((rc = check_ptr(u, g, "u")) || (rc = check_ptr(f, g, "f"))) return rc;
  if (overlap(u, f, (size_t)span_elems(make_geo(*g)) * 8)) return set_error(STENCIL_EINVAL, "u and f overlap");
  return STENCIL_OK;
}

int stencil_smooth_depend(const stencil_grid_t *g, double *u, const double *f, int sweeps,
                          stencil_depend_opts_t *opts, void *stream) {
  int rc = check_fd_uf(g, u, f, "smooth_depend");
  if (rc) return rc;
  return smooth_depend_impl(g, u, f, sweeps, opts, STENCIL_COST_NONE, 0, stream);
}

int stencil_smooth_expensive(const stencil_grid_t *g, double *u, const double *f, int sweeps, int cost_mode,
                             int kmax, stencil_depend_opts_t *depend, void *stream) {
  int rc = check_fd_uf(g, u, f, "smooth_expensive");
  if (rc) return rc;
  if (cost_mode != STENCIL_COST_NONE && cost_mode != STENCIL_COST_UNIFORM && cost_mode != STENCIL_COST_LINEAR)
    return set_error(STENCIL_EINVAL, "smooth_expensive: unknown cost mode");
  if (kmax < 0 || kmax > 100000 || sweeps < 0) return set_error(STENCIL_EINVAL, "smooth_expensive: need 0 <= kmax <= 100000, sweeps >= 0");
  if (depend) return smooth_depend_impl(g, u, f, sweeps, depend, cost_mode, kmax, stream);
  if (sweeps == 0) return STENCIL_OK;
  cudaError_t e = launch_fd_gs_redblack_cost(make_geo(*g), g->dim, u, f, sweeps, cost_mode, kmax,
                                             (cudaStream_t)stream);
  if (e) return set_error(STENCIL_ECUDA, std::string("smooth_expensive: ") + cudaGetErrorString(e));
  return STENCIL_OK;
}

// ------------------------------------------------------------ multigrid

static int check_mg_opts(const stencil_mg_opts_t *o) {
  if (!o) return set_error(STENCIL_EINVAL, "mg: opts is NULL");
  if (o->pre < 0 || o->post < 0 || o->coarse_sweeps < 1 || o->max_levels < 0 || o->max_cycles < 0 ||
      !(o->rel_tol >= 0.0))
    return set_error(STENCIL_EINVAL, "mg: need pre, post, max_levels, max_cycles >= 0, coarse_sweeps >= 1, "
                                     "rel_tol >= 0");
  return STENCIL_OK;
}

// Workspaces and cycle object for one multigrid call on stream s.
static int mg_prepare(const stencil_grid_t *g, const stencil_mg_opts_t *o, cudaStream_t s, MgCycle &cyc,
                      int &levels, double *&dn) {
  const Geo q = make_geo(*g);
  const int maxl = o->max_levels > 0 ? std::min(o->max_levels, MgCycle::kMaxLevels) : MgCycle::kMaxLevels;
  levels = mg_levels(q, g->dim, maxl);
  void *work = levels > 1 ? device_scratch(SCRATCH_MG, mg_work_bytes(q, g->dim, levels), s) : (void *)1;
  void *gsw = device_scratch(SCRATCH_PINGPONG, 3 * (size_t)span_elems(q) * 8, s);
  void *bnd = device_scratch(SCRATCH_BOUNDS, gs_fx_bounds_bytes(), s);
  dn = (double *)device_scratch(SCRATCH_NORMS, 64, s);
  void *red = device_scratch(SCRATCH_REDUCE, mg_reduce_bytes(q, g->dim, levels), s);
  if (!work || !gsw || !bnd || !dn || !red) return set_error(STENCIL_ENOMEM, "mg: workspace allocation failed");
  if (!cyc.setup(q, g->dim, levels, o->pre, o->post, o->coarse_sweeps, work, (double *)gsw, bnd, dn, red, s))
    return set_error(STENCIL_EINVAL, "mg: bad hierarchy");
  return STENCIL_OK;
}

static int mg_check_uf(const stencil_grid_t *g, const double *u, const double *f) {
  int rc = check_grid(g);
  if (rc) return rc;
  if (g->dtype != STENCIL_F64) return set_error(STENCIL_EINVAL, "mg: u and f must be F64");
  if ((rc = require_q1(g, "mg"))) return rc;
  if ((rc = check_ptr(u, g, "u")) || (rc = check_ptr(f, g, "f"))) return rc;
  if (overlap(u, f, (size_t)span_elems(make_geo(*g)) * 8)) return set_error(STENCIL_EINVAL, "u and f overlap");
  return STENCIL_OK;
}

int stencil_mg_vcycle(const stencil_grid_t *g, double *u, const double *f, const stencil_mg_opts_t *opts,
                      void *stream) {
  int rc = mg_check_uf(g, u, f);
  if (rc || (rc = check_mg_opts(opts))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  MgCycle cyc;
  int levels;
  double *dn;
  if ((rc = mg_prepare(g, opts, s, cyc, levels, dn))) return rc;
  cudaError_t e = cyc.run(u, f);
  if (e) return set_error(STENCIL_ECUDA, std::string("mg_vcycle: ") + cudaGetErrorString(e));
  return STENCIL_OK;
}

int stencil_mg_solve(const stencil_grid_t *g, double *u, const double *f, const stencil_mg_opts_t *opts,
                     stencil_mg_info_t *info, void *stream) {
  int rc = mg_check_uf(g, u, f);
  if (rc || (rc = check_mg_opts(opts))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const Geo q = make_geo(*g);
  MgCycle cyc;
  int levels;
  double *dn;
  if ((rc = mg_prepare(g, opts, s, cyc, levels, dn))) return rc;
  double *hn = (double *)host_scratch(64, s);
  // reduction scratch of the convergence test: the cycle's (sized for every level)
  void *red = device_scratch(SCRATCH_REDUCE, mg_reduce_bytes(q, g->dim, levels), s);
  if (!hn || !red) return set_error(STENCIL_ENOMEM, "mg: workspace allocation failed");
  int k = 0;
  double rho = 0.0;
  bool conv = false;
  for (;;) {
    cudaError_t ce = g->dim == 3 ? launch_residual_fx3(q, u, f, nullptr, dn, red, s)
                                 : launch_residual_fx2(q, u, f, nullptr, dn, red, s);
    if (!ce) ce = cudaMemcpyAsync(hn, dn, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (!ce) ce = cudaStreamSynchronize(s);
    if (ce) return set_error(STENCIL_ECUDA, std::string("mg_solve: ") + cudaGetErrorString(ce));
    rho = hn[1] > 0.0 ? std::sqrt(hn[0]) / std::sqrt(hn[1]) : std::sqrt(hn[0]);
    if (info && info->relres_history) info->relres_history[k] = rho;
    if (rho <= opts->rel_tol) {
      conv = true;
      break;
    }
    if (k >= opts->max_cycles) break;
    ce = cyc.run(u, f);
    if (ce) return set_error(STENCIL_ECUDA, std::string("mg_solve: ") + cudaGetErrorString(ce));
    ++k;
  }
  if (info) {
    info->cycles = k;
    info->converged = conv ? 1 : 0;
    info->levels = levels;
    info->relres = rho;
  }
  if (!conv) return set_error(STENCIL_ENOTCONV, "mg_solve: max_cycles reached before rel_tol");
  return STENCIL_OK;
}

static int check_transfer(const stencil_grid_t *fine, const stencil_grid_t *coarse) {
  int rc = check_grid(fine);
  if (rc || (rc = check_grid(coarse))) return rc;
  if (fine->dtype != STENCIL_F64 || coarse->dtype != STENCIL_F64)
    return set_error(STENCIL_EINVAL, "mg transfer: F64 only");
  if (fine->dim != coarse->dim) return set_error(STENCIL_EINVAL, "mg transfer: dim mismatch");
  if ((rc = require_q1(fine, "mg transfer")) || (rc = require_q1(coarse, "mg transfer"))) return rc;
  Geo qc;
  if (!mg_coarse(make_geo(*fine), fine->dim, qc))
    return set_error(STENCIL_EINVAL, "mg transfer: the fine grid has no coarse grid");
  if (coarse->n[0] != qc.nx || coarse->n[1] != qc.ny || (fine->dim == 3 && coarse->n[2] != qc.nz))
    return set_error(STENCIL_EINVAL, "mg transfer: coarse n must be the hierarchy's coarse grid of the fine n");
  return STENCIL_OK;
}

int stencil_mg_restrict(const stencil_grid_t *fine, const double *rf, const stencil_grid_t *coarse, double *rc,
                        void *stream) {
  int r = check_transfer(fine, coarse);
  if (r || (r = check_ptr(rf, fine, "rf")) || (r = check_ptr(rc, coarse, "rc"))) return r;
  const Geo qf = make_geo(*fine), qc = make_geo(*coarse);
  const size_t bf = (size_t)span_elems(qf) * 8, bc = (size_t)span_elems(qc) * 8;
  if ((const char *)rf < (const char *)rc + bc && (const char *)rc < (const char *)rf + bf)
    return set_error(STENCIL_EINVAL, "rf and rc overlap");
  cudaError_t e = launch_mg_restrict(qf, qc, fine->dim, rf, rc, (cudaStream_t)stream);
  if (e) return set_error(STENCIL_ECUDA, std::string("mg_restrict: ") + cudaGetErrorString(e));
  return STENCIL_OK;
}

int stencil_mg_prolong_add(const stencil_grid_t *fine, double *uf, const stencil_grid_t *coarse, const double *ec,
                           void *stream) {
  int r = check_transfer(fine, coarse);
  if (r || (r = check_ptr(uf, fine, "uf")) || (r = check_ptr(ec, coarse, "ec"))) return r;
  const Geo qf = make_geo(*fine), qc = make_geo(*coarse);
  const size_t bf = (size_t)span_elems(qf) * 8, bc = (size_t)span_elems(qc) * 8;
  if ((const char *)ec < (const char *)uf + bf && (const char *)uf < (const char *)ec + bc)
    return set_error(STENCIL_EINVAL, "uf and ec overlap");
  cudaError_t e = launch_mg_prolong_add(qf, qc, fine->dim, ec, uf, (cudaStream_t)stream);
  if (e) return set_error(STENCIL_ECUDA, std::string("mg_prolong_add: ") + cudaGetErrorString(e));
  return STENCIL_OK;
}

}  // extern "C"
