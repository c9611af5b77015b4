// Request server with continuous batching (stencil_server_*).
//
// A host engine thread owns every admitted request's device state.  Requests wait in a
// FIFO; the engine admits them (looking past a blocked head at the next few) whenever
// the request's device footprint fits the HBM budget and an in-flight slot is free,
// allocates its buffers stream-ordered, and drives it on one of several CUDA streams:
//   SMOOTH: `sweeps` coloured Gauss-Seidel sweeps (the FP64 fixed-point kernels);
//   SOLVE:  iterative refinement, one correction per step (residual and norms in FP64,
//           inner coloured GS sweeps in FP32 / bf16 / FP64), or (solver MG) one FP64
//           multigrid V-cycle per step; the norm is read back asynchronously and the
//           next step is issued once it has arrived.
// Work of different requests is on different streams and overlaps on the device; new
// requests join as soon as memory and slots free up.  Each request uses only its own
// buffers and deterministic kernels, so its result does not depend on what else runs.
// Results stay resident until fetched or released.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace stencil {
namespace {

// SplitMix64 (Steele, Lea, Flood 2014) used as a counter-based generator: element i of
// the stream with seed s is mix(s + (i + 1) * 0x9E3779B97F4A7C15), mapped to a double in
// [-1, 1) from its top 53 bits.
__host__ __device__ __forceinline__ unsigned long long splitmix_mix(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_fill_rhs(double *f, int n, unsigned long long seed) {
  const int64_t W = n + 1, total = W * W * W;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = i % W, y = (i / W) % W, z = i / (W * W);
    const bool inner = x > 0 && x < n && y > 0 && y < n && z > 0 && z < n;
    const unsigned long long r = splitmix_mix(seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull);
    f[i] = inner ? ((double)(r >> 11) * 0x1p-53) * 2.0 - 1.0 : 0.0;
  }
}

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

enum Phase { P_PENDING, P_RUNNING, P_DONE };

struct Req {
  uint64_t ticket = 0;
  stencil_request_t r{};
  std::vector<double> f_host, u_host;  // copies made at submit (empty: generated / zeros)
  uint64_t seed = 0;
  bool seeded = false;
  Phase phase = P_PENDING;
  int stream = 0;
  size_t footprint = 0;
  Geo q{};
  // device state
  double *u = nullptr, *f = nullptr, *work = nullptr, *norms = nullptr;
  void *bounds = nullptr, *red = nullptr, *rlo = nullptr, *elo = nullptr, *wlo = nullptr;
  double *hnorms = nullptr;  // pinned, 2 doubles (a slot of the server's pool)
  int hslot = -1;
  void *mgw = nullptr;  // multigrid: coarse-level arrays
  MgCycle cyc;          // multigrid: the request's V-cycle
  cudaEvent_t ev = nullptr;
  bool step_in_flight = false;
  int iterations = 0;
  double relres = 0.0;
  int status = STENCIL_OK;
  double t_submit = 0, t_admit = 0, t_done = 0;
};

}  // namespace
}  // namespace stencil

using namespace stencil;

struct stencil_server {
  size_t budget = 0, used = 0;
  stencil_server_opts_t o{};
  int device = 0;
  std::vector<cudaStream_t> streams;
  cudaMemPool_t pool = nullptr;
  std::mutex mu;
  std::condition_variable cv_done, cv_work;
  std::deque<uint64_t> pending;
  std::map<uint64_t, Req *> reqs;
  // admitted requests not yet finished: the engine polls only these, so results that
  // stay resident until released cost it nothing
  std::vector<Req *> running;
  uint64_t next_ticket = 1;
  int inflight = 0;
  int next_stream = 0;
  bool stop = false;
  std::thread engine;
  std::chrono::steady_clock::time_point t0;
  stencil_server_stats_t stats{};
  std::string engine_error;
  double *hpool = nullptr;       // pinned norms, 8 doubles per in-flight slot
  std::vector<int> hfree;        // free slots of hpool
};

namespace {

size_t elem_bytes(int dtype) { return dtype == STENCIL_F64 ? 8 : (dtype == STENCIL_F32 ? 4 : 2); }

size_t footprint_of(const stencil_server_opts_t &o, const stencil_request_t &r, Geo &q) {
  stencil_grid_t g{};
  g.dim = 3;
  g.dtype = STENCIL_F64;
  g.n[0] = g.n[1] = g.n[2] = r.n;
  g.h = 1.0 / r.n;
  q = make_geo(g);
  const size_t span = (size_t)span_elems(q);
  size_t b = 2 * span * 8 + 64 + 256;  // u, f, norms
  if (r.kind == STENCIL_REQ_SMOOTH) {
    b += 3 * span * 8 + gs_fx_bounds_bytes();
  } else if (o.solver == STENCIL_SOLVER_MG) {
    const int L = mg_levels(q, 3, MgCycle::kMaxLevels);
    b += mg_work_bytes(q, 3, L) + mg_reduce_bytes(q, 3, L) + 3 * span * 8 + gs_fx_bounds_bytes();
  } else {
    const size_t e = elem_bytes(o.inner_dtype);
    b += ops_fx_reduce_bytes(q) + 2 * span * e;  // residual and correction in the inner type
    b += o.inner_dtype == STENCIL_F64 ? 3 * span * 8 + gs_fx_bounds_bytes() : span * e;
  }
  return b;
}

cudaError_t dalloc(stencil_server *s, void **p, size_t bytes, cudaStream_t st) {
  return cudaMallocFromPoolAsync(p, bytes, s->pool, st);
}

void release_device(stencil_server *s, Req *q) {
  cudaStream_t st = s->streams[q->stream];
  void *ptrs[] = {q->u, q->f, q->work, q->norms, q->bounds, q->red, q->rlo, q->elo, q->wlo, q->mgw};
  for (void *p : ptrs)
    if (p) cudaFreeAsync(p, st);
  q->u = q->f = q->work = q->norms = nullptr;
  q->bounds = q->red = q->rlo = q->elo = q->wlo = q->mgw = nullptr;
  if (q->hslot >= 0) {
    s->hfree.push_back(q->hslot);
    q->hslot = -1;
    q->hnorms = nullptr;
  }
  if (q->ev) {
    cudaEventDestroy(q->ev);
    q->ev = nullptr;
  }
}

// Issue the residual of a SOLVE request and the read-back of its norms.
cudaError_t issue_residual(stencil_server *s, Req *q) {
  cudaStream_t st = s->streams[q->stream];
  const int kind = s->o.inner_dtype == STENCIL_F64 ? 0 : (s->o.inner_dtype == STENCIL_F32 ? 1 : 2);
  cudaError_t e = s->o.solver == STENCIL_SOLVER_MG
                      ? launch_residual_fx3(q->q, q->u, q->f, nullptr, q->norms, q->red, st, 0)
                      : launch_residual_fx3(q->q, q->u, q->f, (double *)q->rlo, q->norms, q->red, st, kind);
  if (!e) e = cudaMemcpyAsync(q->hnorms, q->norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaEventRecord(q->ev, st);
  q->step_in_flight = true;
  return e;
}

cudaError_t issue_correction(stencil_server *s, Req *q) {
  if (s->o.solver == STENCIL_SOLVER_MG) return q->cyc.run(q->u, q->f);
  cudaStream_t st = s->streams[q->stream];
  const size_t span = (size_t)span_elems(q->q);
  const int dt = s->o.inner_dtype;
  cudaError_t e = cudaMemsetAsync(q->elo, 0, span * elem_bytes(dt), st);
  if (!e) {
    if (dt == STENCIL_F64)
      e = launch_gs_sweeps_fx3(q->q, (double *)q->elo, (const double *)q->rlo, s->o.inner_sweeps,
                               (double *)q->wlo, q->bounds, st);
    else if (dt == STENCIL_F32)
      e = launch_gs_sweeps_f32_3d(q->q, (float *)q->elo, (const float *)q->rlo, s->o.inner_sweeps, (float *)q->wlo, st);
    else
      e = launch_gs_sweeps_bf16_3d(q->q, q->elo, q->rlo, s->o.inner_sweeps, q->wlo, st);
  }
  if (!e) e = launch_add_correction(q->q, 3, q->u, q->elo, dt, st);
  return e;
}

// Allocate and initialise an admitted request; queue its first step.
// Called with the server's mutex held: the request's stream and pinned norms slot.
void assign_slots(stencil_server *s, Req *q) {
  q->stream = s->next_stream;
  s->next_stream = (s->next_stream + 1) % (int)s->streams.size();
  q->hslot = s->hfree.back();
  s->hfree.pop_back();
  q->hnorms = s->hpool + 8 * q->hslot;
}

// Called without the mutex: only the engine thread touches a running request's
// buffers, and the allocator and streams are thread-safe.
cudaError_t admit(stencil_server *s, Req *q) {
  cudaStream_t st = s->streams[q->stream];
  const size_t span = (size_t)span_elems(q->q);
  cudaError_t e = cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming);
  if (!e) e = dalloc(s, (void **)&q->u, span * 8, st);
  if (!e) e = dalloc(s, (void **)&q->f, span * 8, st);
  if (!e) e = dalloc(s, (void **)&q->norms, 64, st);
  if (e) return e;
  if (!q->u_host.empty())
    e = cudaMemcpyAsync(q->u, q->u_host.data(), span * 8, cudaMemcpyHostToDevice, st);
  else
    e = cudaMemsetAsync(q->u, 0, span * 8, st);
  if (!e) {
    if (q->seeded)
      k_fill_rhs<<<1216, 256, 0, st>>>(q->f, q->r.n, q->seed), e = cudaGetLastError();
    else
      e = cudaMemcpyAsync(q->f, q->f_host.data(), span * 8, cudaMemcpyHostToDevice, st);
  }
  if (e) return e;
  if (q->r.kind == STENCIL_REQ_SMOOTH) {
    e = dalloc(s, (void **)&q->work, 3 * span * 8, st);
    if (!e) e = dalloc(s, &q->bounds, gs_fx_bounds_bytes(), st);
    if (!e && q->r.sweeps > 0) e = launch_gs_sweeps_fx3(q->q, q->u, q->f, q->r.sweeps, q->work, q->bounds, st);
    if (!e) e = cudaEventRecord(q->ev, st);
    q->step_in_flight = true;
  } else if (s->o.solver == STENCIL_SOLVER_MG) {
    const int L = mg_levels(q->q, 3, MgCycle::kMaxLevels);
    const size_t rb = mg_reduce_bytes(q->q, 3, L);
    e = dalloc(s, &q->red, rb, st);
    if (!e) e = cudaMemsetAsync(q->red, 0, rb, st);
    if (!e) e = dalloc(s, &q->mgw, mg_work_bytes(q->q, 3, L) + 256, st);
    if (!e) e = dalloc(s, (void **)&q->work, 3 * span * 8, st);
    if (!e) e = dalloc(s, &q->bounds, gs_fx_bounds_bytes(), st);
    if (!e && !q->cyc.setup(q->q, 3, L, 2, 2, 20, q->mgw, q->work, q->bounds, q->norms, q->red, st))
      e = cudaErrorInvalidValue;
    if (!e) e = issue_residual(s, q);
  } else {
    const size_t eb = elem_bytes(s->o.inner_dtype);
    e = dalloc(s, &q->red, ops_fx_reduce_bytes(q->q), st);
    if (!e) e = cudaMemsetAsync(q->red, 0, ops_fx_reduce_bytes(q->q), st);
    if (!e) e = dalloc(s, &q->rlo, span * eb, st);
    if (!e) e = dalloc(s, &q->elo, span * eb, st);
    if (!e) {
      if (s->o.inner_dtype == STENCIL_F64) {
        e = dalloc(s, &q->wlo, 3 * span * 8, st);
        if (!e) e = dalloc(s, &q->bounds, gs_fx_bounds_bytes(), st);
      } else {
        e = dalloc(s, &q->wlo, span * eb, st);
      }
    }
    if (!e) e = issue_residual(s, q);
  }
  return e;
}

void finish(stencil_server *s, Req *q, int status) {
  q->status = status;
  q->phase = P_DONE;
  q->t_done = now_s(s->t0);
  q->step_in_flight = false;
  // working buffers go back at once; u stays resident for fetch
  cudaStream_t st = s->streams[q->stream];
  void *ptrs[] = {q->f, q->work, q->norms, q->bounds, q->red, q->rlo, q->elo, q->wlo, q->mgw};
  for (void *p : ptrs)
    if (p) cudaFreeAsync(p, st);
  q->f = q->work = q->norms = nullptr;
  q->bounds = q->red = q->rlo = q->elo = q->wlo = q->mgw = nullptr;
  if (q->hslot >= 0) {
    s->hfree.push_back(q->hslot);
    q->hslot = -1;
    q->hnorms = nullptr;
  }
  const size_t resident = (size_t)span_elems(q->q) * 8;
  s->used -= q->footprint - resident;
  q->footprint = resident;
  --s->inflight;
  s->stats.completed++;
}

// The engine thread.  The mutex guards the queues, the budget, the counters and the
// phase of every request; it is held for that bookkeeping only, never across kernel
// launches, allocations or event queries, so submissions, polls and releases from
// client threads are not held up by the device work being issued.
void engine_loop(stencil_server *s) {
  cudaSetDevice(s->device);
  std::vector<Req *> admitted, run, done;
  std::vector<int> done_status;
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    bool progress = false;
    // admission (FIFO, looking past a blocked head at the next few requests)
    admitted.clear();
    int looked = 0;
    for (auto it = s->pending.begin(); it != s->pending.end() && looked < 16;) {
      Req *q = s->reqs[*it];
      ++looked;
      if (s->inflight < s->o.max_inflight && s->used + q->footprint <= s->budget) {
        s->used += q->footprint;
        ++s->inflight;
        q->phase = P_RUNNING;
        q->t_admit = now_s(s->t0);
        assign_slots(s, q);
        admitted.push_back(q);
        it = s->pending.erase(it);
      } else {
        ++it;
      }
    }
    run = s->running;
    lk.unlock();
    // device work, without the mutex
    done.clear();
    done_status.clear();
    for (Req *q : admitted) {
      progress = true;
      cudaError_t e = admit(s, q);
      if (e) {
        std::lock_guard<std::mutex> g(s->mu);
        s->engine_error = cudaGetErrorString(e);
        done.push_back(q);
        done_status.push_back(STENCIL_ECUDA);
      } else {
        run.push_back(q);
      }
    }
    for (Req *q : run) {
      if (!q->step_in_flight) continue;
      const cudaError_t qe = cudaEventQuery(q->ev);
      if (qe == cudaErrorNotReady) continue;
      progress = true;
      q->step_in_flight = false;
      int status = 1;  // 1: keep running
      if (qe != cudaSuccess) {
        std::lock_guard<std::mutex> g(s->mu);
        s->engine_error = cudaGetErrorString(qe);
        status = STENCIL_ECUDA;
      } else if (q->r.kind == STENCIL_REQ_SMOOTH) {
        q->iterations = q->r.sweeps;
        status = STENCIL_OK;
      } else {
        const double rr = q->hnorms[0], ff = q->hnorms[1];
        q->relres = ff > 0.0 ? std::sqrt(rr) / std::sqrt(ff) : std::sqrt(rr);
        if (q->relres <= q->r.rel_tol || q->iterations >= s->o.max_outer) {
          status = q->relres <= q->r.rel_tol ? STENCIL_OK : STENCIL_ENOTCONV;
        } else {
          cudaError_t e = issue_correction(s, q);
          ++q->iterations;
          if (!e) e = issue_residual(s, q);
          if (e) {
            std::lock_guard<std::mutex> g(s->mu);
            s->engine_error = cudaGetErrorString(e);
            status = STENCIL_ECUDA;
          }
        }
      }
      if (status != 1) {
        done.push_back(q);
        done_status.push_back(status);
      }
    }
    lk.lock();
    for (Req *q : admitted)
      if (q->phase == P_RUNNING) s->running.push_back(q);
    for (size_t i = 0; i < done.size(); ++i) finish(s, done[i], done_status[i]);
    if (!done.empty()) {
      s->running.erase(std::remove_if(s->running.begin(), s->running.end(),
                                      [](const Req *q) { return q->phase != P_RUNNING; }),
                       s->running.end());
      s->cv_done.notify_all();
    }
    if (!progress) {
      // nothing to do right now: wait for a submission, or poll the GPU again shortly
      s->cv_work.wait_for(lk, std::chrono::microseconds(s->inflight ? 20 : 2000));
    }
  }
}

Req *find(stencil_server *s, uint64_t t) {
  auto it = s->reqs.find(t);
  return it == s->reqs.end() ? nullptr : it->second;
}

void fill_result(const Req *q, stencil_result_t *res) {
  if (!res) return;
  res->status = q->status;
  res->iterations = q->iterations;
  res->relres = q->relres;
  res->t_submit = q->t_submit;
  res->t_admit = q->t_admit;
  res->t_done = q->t_done;
}

}  // namespace

extern "C" {

int stencil_server_create(size_t hbm_budget_bytes, const stencil_server_opts_t *opts, stencil_server_t **out) {
  if (!out) return set_error(STENCIL_EINVAL, "server_create: out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes == 0) return set_error(STENCIL_EINVAL, "server_create: zero budget");
  stencil_server *s = new stencil_server();
  s->budget = hbm_budget_bytes;
  stencil_server_opts_t o{};
  if (opts) o = *opts;
  if (o.streams <= 0) o.streams = 8;
  if (o.max_inflight <= 0) o.max_inflight = 64;
  if (o.inner_sweeps <= 0) o.inner_sweeps = 8;
  if (o.inner_dtype != STENCIL_F64 && o.inner_dtype != STENCIL_BF16) o.inner_dtype = STENCIL_F32;
  if (o.max_outer <= 0) o.max_outer = 100000;
  if (o.solver != STENCIL_SOLVER_REFINE && o.solver != STENCIL_SOLVER_MG) {
    delete s;
    return set_error(STENCIL_EINVAL, "server_create: unknown solver");
  }
  s->o = o;
  cudaGetDevice(&s->device);
  s->t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaDeviceGetDefaultMemPool(&s->pool, s->device);
  if (!e) {
    uint64_t thr = UINT64_MAX;  // keep freed memory in the pool for reuse
    e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  if (!e) e = cudaMallocHost(&s->hpool, (size_t)o.max_inflight * 8 * sizeof(double));
  for (int i = 0; i < o.max_inflight; ++i) s->hfree.push_back(o.max_inflight - 1 - i);
  for (int i = 0; i < o.streams && !e; ++i) {
    cudaStream_t st;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (!e) s->streams.push_back(st);
  }
  if (e) {
    for (auto st : s->streams) cudaStreamDestroy(st);
    if (s->hpool) cudaFreeHost(s->hpool);
    delete s;
    return set_error(STENCIL_ECUDA, std::string("server_create: ") + cudaGetErrorString(e));
  }
  s->engine = std::thread(engine_loop, s);
  *out = s;
  return STENCIL_OK;
}

int stencil_server_submit(stencil_server_t *s, const stencil_request_t *r, uint64_t *ticket) {
  if (!s || !r || !ticket) return set_error(STENCIL_EINVAL, "server_submit: NULL argument");
  if (r->kind != STENCIL_REQ_SMOOTH && r->kind != STENCIL_REQ_SOLVE)
    return set_error(STENCIL_EINVAL, "server_submit: unknown request kind");
  if (r->n < 2 || r->n > 2048) return set_error(STENCIL_EINVAL, "server_submit: n must be in [2, 2048]");
  if (r->kind == STENCIL_REQ_SMOOTH && r->sweeps < 0) return set_error(STENCIL_EINVAL, "server_submit: sweeps < 0");
  if (r->kind == STENCIL_REQ_SOLVE && !(r->rel_tol >= 0.0)) return set_error(STENCIL_EINVAL, "server_submit: rel_tol");
  Req *q = new Req();
  q->r = *r;
  q->footprint = footprint_of(s->o, *r, q->q);
  if (q->footprint > s->budget) {
    delete q;
    return set_error(STENCIL_EADMIT, "server_submit: request footprint exceeds the HBM budget");
  }
  const size_t span = (size_t)span_elems(q->q);
  if (r->f) {
    q->f_host.assign(r->f, r->f + span);
  } else {
    q->seeded = true;
    q->seed = (uint64_t)r->f_seed;
  }
  if (r->u0) q->u_host.assign(r->u0, r->u0 + span);
  std::lock_guard<std::mutex> lk(s->mu);
  q->ticket = s->next_ticket++;
  q->t_submit = now_s(s->t0);
  s->reqs[q->ticket] = q;
  s->pending.push_back(q->ticket);
  s->stats.submitted++;
  *ticket = q->ticket;
  s->cv_work.notify_one();
  return STENCIL_OK;
}

int stencil_server_poll(stencil_server_t *s, uint64_t ticket, stencil_result_t *res) {
  if (!s) return set_error(STENCIL_EINVAL, "server_poll: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  Req *q = find(s, ticket);
  if (!q) return set_error(STENCIL_ENOTFOUND, "server_poll: unknown ticket");
  if (q->phase != P_DONE) return STENCIL_EBUSY;
  fill_result(q, res);
  return STENCIL_OK;
}

int stencil_server_wait(stencil_server_t *s, uint64_t ticket, int64_t timeout_us, stencil_result_t *res) {
  if (!s) return set_error(STENCIL_EINVAL, "server_wait: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  Req *q = find(s, ticket);
  if (!q) return set_error(STENCIL_ENOTFOUND, "server_wait: unknown ticket");
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
  while (q->phase != P_DONE) {
    if (timeout_us >= 0 && s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && q->phase != P_DONE)
      return set_error(STENCIL_ETIMEDOUT, "server_wait: timed out");
    if (timeout_us < 0) s->cv_done.wait(lk);
  }
  fill_result(q, res);
  return STENCIL_OK;
}

int stencil_server_fetch(stencil_server_t *s, uint64_t ticket, double *u_host) {
  if (!s || !u_host) return set_error(STENCIL_EINVAL, "server_fetch: NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  Req *q = find(s, ticket);
  if (!q) return set_error(STENCIL_ENOTFOUND, "server_fetch: unknown ticket");
  if (q->phase != P_DONE) return STENCIL_EBUSY;
  if (q->status == STENCIL_ECUDA) return set_error(STENCIL_ECUDA, "server_fetch: request failed: " + s->engine_error);
  cudaStream_t st = s->streams[q->stream];
  const size_t bytes = (size_t)span_elems(q->q) * 8;
  double *u = q->u;
  lk.unlock();  // the copy does not need the lock; the request is done and stays put
  cudaError_t e = cudaMemcpyAsync(u_host, u, bytes, cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) return set_error(STENCIL_ECUDA, std::string("server_fetch: ") + cudaGetErrorString(e));
  return stencil_server_release(s, ticket);
}

int stencil_server_release(stencil_server_t *s, uint64_t ticket) {
  if (!s) return set_error(STENCIL_EINVAL, "server_release: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  Req *q = find(s, ticket);
  if (!q) return set_error(STENCIL_ENOTFOUND, "server_release: unknown ticket");
  if (q->phase != P_DONE) return STENCIL_EBUSY;
  release_device(s, q);
  s->used -= q->footprint;
  s->reqs.erase(ticket);
  delete q;
  s->cv_work.notify_one();
  return STENCIL_OK;
}

int stencil_server_stats(stencil_server_t *s, stencil_server_stats_t *st) {
  if (!s || !st) return set_error(STENCIL_EINVAL, "server_stats: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *st = s->stats;
  st->pending = (int64_t)s->pending.size();
  st->inflight = s->inflight;
  st->hbm_used = s->used;
  st->hbm_budget = s->budget;
  return STENCIL_OK;
}

int stencil_server_destroy(stencil_server_t *s) {
  if (!s) return STENCIL_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  s->engine.join();
  cudaDeviceSynchronize();
  for (auto &kv : s->reqs) {
    release_device(s, kv.second);
    delete kv.second;
  }
  for (auto st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  cudaFreeHost(s->hpool);
  delete s;
  return STENCIL_OK;
}

}  // extern "C"
