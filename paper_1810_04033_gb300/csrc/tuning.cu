// Launch-shape autotuner and its cache: for a grid shape and a call, time the
// candidate chunkings (3D: planes per CTA of the plane-streaming kernels; 2D: rows per
// warp, and for the multi-sweep smoothers the number of sweeps per pass over memory)
// on scratch arrays, keep the fastest in a per-process table that the launchers
// consult, and save or load that table as JSON.
//
// The paper tunes nothing of this kind; its tiling and colour-fusion discussion
// (Sections 5 and 6) motivates choosing the tile depth and the fusion depth per grid.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <cctype>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

namespace stencil {
namespace {

// ------------------------------------------------------------ the table
using Key = std::tuple<std::string, int, int, int64_t, int64_t, int64_t, int64_t>;  // device, call, dim, n, pitch

struct Entry {
  int chunk = 0, depth = 0;
  double ms = 0.0;
};

std::mutex g_mu;
std::map<Key, Entry> g_table;
std::atomic<size_t> g_count{0};
std::once_flag g_env_once;

std::string device_name() {
  static std::mutex mu;
  static std::string names[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return std::string("unknown");
  std::lock_guard<std::mutex> lk(mu);
  if (names[dev].empty()) {
    cudaDeviceProp p;
    names[dev] = cudaGetDeviceProperties(&p, dev) == cudaSuccess ? std::string(p.name) : std::string("unknown");
  }
  return names[dev];
}

Key make_key(const std::string &dev, int call, const Geo &q) {
  const int dim = q.nz == 0 ? 2 : 3;
  return Key(dev, call, dim, q.nx, q.ny, q.nz, q.pitch);
}

bool tunable_call(int call) {
  return call == STENCIL_CALL_SMOOTH_COLOURED || call == STENCIL_CALL_SMOOTH_JACOBI ||
         call == STENCIL_CALL_APPLY_ELEMENTWISE || call == STENCIL_CALL_APPLY_STENCIL;
}

void put(const Key &k, const Entry &e) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_table[k] = e;
  g_count.store(g_table.size(), std::memory_order_release);
}

void erase(const Key &k) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_table.erase(k);
  g_count.store(g_table.size(), std::memory_order_release);
}

bool get(const Key &k, Entry &e) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_table.find(k);
  if (it == g_table.end()) return false;
  e = it->second;
  return true;
}

// ------------------------------------------------------------ JSON (the subset written here)
struct JVal {
  enum Kind { NUL, NUM, STR, ARR, OBJ, BOOL } kind = NUL;
  double num = 0.0;
  std::string str;
  std::vector<JVal> arr;
  std::vector<std::pair<std::string, JVal>> obj;
  const JVal *field(const char *name) const {
    for (auto &kv : obj)
      if (kv.first == name) return &kv.second;
    return nullptr;
  }
};

struct JParser {
  const char *p, *end;
  bool ok = true;
  void ws() {
    while (p < end && std::isspace((unsigned char)*p)) ++p;
  }
  bool lit(const char *w) {
    size_t n = strlen(w);
    if ((size_t)(end - p) >= n && strncmp(p, w, n) == 0) {
      p += n;
      return true;
    }
    return false;
  }
  std::string string() {
    std::string out;
    ++p;  // opening quote
    while (p < end && *p != '"') {
      char c = *p++;
      if (c == '\\' && p < end) {
        char e = *p++;
        c = e == 'n' ? '\n' : e == 't' ? '\t' : e;  // \" \\ \/ and the rest taken literally
      }
      out.push_back(c);
    }
    if (p >= end) ok = false;
    else ++p;
    return out;
  }
  JVal value(int depth) {
    JVal v;
    ws();
    if (p >= end || depth > 16) {
      ok = false;
      return v;
    }
    if (*p == '{') {
      v.kind = JVal::OBJ;
      ++p;
      ws();
      if (p < end && *p == '}') {
        ++p;
        return v;
      }
      while (ok) {
        ws();
        if (p >= end || *p != '"') {
          ok = false;
          break;
        }
        std::string k = string();
        ws();
        if (p >= end || *p != ':') {
          ok = false;
          break;
        }
        ++p;
        v.obj.emplace_back(k, value(depth + 1));
        ws();
        if (p < end && *p == ',') {
          ++p;
          continue;
        }
        if (p < end && *p == '}') {
          ++p;
          break;
        }
        ok = false;
      }
    } else if (*p == '[') {
      v.kind = JVal::ARR;
      ++p;
      ws();
      if (p < end && *p == ']') {
        ++p;
        return v;
      }
      while (ok) {
        v.arr.push_back(value(depth + 1));
        ws();
        if (p < end && *p == ',') {
          ++p;
          continue;
        }
        if (p < end && *p == ']') {
          ++p;
          break;
        }
        ok = false;
      }
    } else if (*p == '"') {
      v.kind = JVal::STR;
      v.str = string();
    } else if (lit("true")) {
      v.kind = JVal::BOOL;
      v.num = 1;
    } else if (lit("false")) {
      v.kind = JVal::BOOL;
    } else if (lit("null")) {
      v.kind = JVal::NUL;
    } else {
      char *e = nullptr;
      v.num = strtod(p, &e);
      if (e == p) ok = false;
      v.kind = JVal::NUM;
      p = e ? e : p;
    }
    return v;
  }
};

std::string json_escape(const std::string &s) {
  std::string o;
  for (char c : s) {
    if (c == '"' || c == '\\') o.push_back('\\');
    if ((unsigned char)c >= 0x20) o.push_back(c);
  }
  return o;
}

void load_env_cache();

int save_table(const char *path) {
  std::vector<std::pair<Key, Entry>> rows;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    rows.assign(g_table.begin(), g_table.end());
  }
  std::string tmp = std::string(path) + ".tmp";
  FILE *fp = fopen(tmp.c_str(), "w");
  if (!fp) return set_error(STENCIL_EINVAL, std::string("tuning_save: cannot write ") + tmp);
  fprintf(fp, "{\"format\": \"stencil_gb300_tuning\", \"version\": 1, \"entries\": [");
  for (size_t i = 0; i < rows.size(); ++i) {
    const Key &k = rows[i].first;
    const Entry &e = rows[i].second;
    fprintf(fp,
            "%s\n  {\"device\": \"%s\", \"call\": %d, \"dim\": %d, \"n\": [%lld, %lld, %lld], \"pitch\": %lld, "
            "\"chunk\": %d, \"depth\": %d, \"ms\": %.6g}",
            i ? "," : "", json_escape(std::get<0>(k)).c_str(), std::get<1>(k), std::get<2>(k),
            (long long)std::get<3>(k), (long long)std::get<4>(k), (long long)std::get<5>(k),
            (long long)std::get<6>(k), e.chunk, e.depth, e.ms);
  }
  fprintf(fp, "\n]}\n");
  const bool ok = fflush(fp) == 0;
  fclose(fp);
  if (!ok || rename(tmp.c_str(), path) != 0) {
    remove(tmp.c_str());
    return set_error(STENCIL_EINVAL, std::string("tuning_save: cannot write ") + path);
  }
  return STENCIL_OK;
}

// Reads a file written by save_table; all entries or none are added.
int load_table(const char *path) {
  FILE *fp = fopen(path, "rb");
  if (!fp) return set_error(STENCIL_EINVAL, std::string("tuning_load: cannot read ") + path);
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof buf, fp)) > 0 && text.size() < (64u << 20)) text.append(buf, n);
  fclose(fp);
  JParser jp{text.data(), text.data() + text.size()};
  JVal root = jp.value(0);
  const JVal *fmt = root.kind == JVal::OBJ ? root.field("format") : nullptr;
  const JVal *ent = root.kind == JVal::OBJ ? root.field("entries") : nullptr;
  if (!jp.ok || !fmt || fmt->str != "stencil_gb300_tuning" || !ent || ent->kind != JVal::ARR)
    return set_error(STENCIL_EINVAL, std::string("tuning_load: not a tuning cache: ") + path);
  std::vector<std::pair<Key, Entry>> rows;
  for (const JVal &e : ent->arr) {
    const JVal *dev = e.field("device"), *call = e.field("call"), *dim = e.field("dim"), *nn = e.field("n"),
               *pitch = e.field("pitch"), *chunk = e.field("chunk"), *depth = e.field("depth"), *ms = e.field("ms");
    if (!dev || dev->kind != JVal::STR || !call || !dim || !nn || nn->kind != JVal::ARR || nn->arr.size() != 3 ||
        !pitch || !chunk || !depth || !tunable_call((int)call->num) || (dim->num != 2 && dim->num != 3) ||
        chunk->num < 0 || chunk->num > 4096 || depth->num < 0 || depth->num > 2)
      return set_error(STENCIL_EINVAL, std::string("tuning_load: malformed entry in ") + path);
    Entry x;
    x.chunk = (int)chunk->num;
    x.depth = (int)depth->num;
    x.ms = ms ? ms->num : 0.0;
    rows.emplace_back(Key(dev->str, (int)call->num, (int)dim->num, (int64_t)nn->arr[0].num, (int64_t)nn->arr[1].num,
                          (int64_t)nn->arr[2].num, (int64_t)pitch->num),
                      x);
  }
  for (auto &r : rows) put(r.first, r.second);
  return STENCIL_OK;
}

void load_env_cache() {
  const char *path = getenv("STENCIL_TUNING_CACHE");
  if (!path || !*path) return;
  FILE *fp = fopen(path, "rb");
  if (!fp) return;  // no cache yet: nothing to consult
  fclose(fp);
  load_table(path);
}

// ------------------------------------------------------------ timing candidates
// Deterministic scratch inputs in [-1, 1) (SplitMix64 of the element index; Steele,
// Lea and Flood 2014), zero on the boundary and in the row padding.
__global__ void k_tune_fill(double *a, Geo q, int dim, unsigned long long seed) {
  const int64_t span = q.plane * (q.nz + 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < span; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = i % q.pitch, y = (i / q.pitch) % (q.ny + 1), z = i / q.plane;
    const bool in = x >= 1 && x < q.nx && y >= 1 && y < q.ny && (dim == 2 || (z >= 1 && z < q.nz));
    unsigned long long v = seed + 0x9e3779b97f4a7c15ull * (unsigned long long)(i + 1);
    v = (v ^ (v >> 30)) * 0xbf58476d1ce4e5b9ull;
    v = (v ^ (v >> 27)) * 0x94d049bb133111ebull;
    v ^= v >> 31;
    a[i] = (x <= q.nx && in) ? (double)(v >> 11) * 0x1p-52 - 1.0 : 0.0;
  }
}

struct Candidate {
  int chunk, depth;
};

std::vector<Candidate> candidates(int call, int dim) {
  std::vector<Candidate> c;
  if (dim == 3) {
    const int lo = call == STENCIL_CALL_SMOOTH_COLOURED ? 2 : 4;
    const int hi = call == STENCIL_CALL_SMOOTH_COLOURED ? 16 : 32;
    for (int cz = lo; cz <= hi; cz *= 2) c.push_back({cz, 0});
  } else if (call == STENCIL_CALL_APPLY_ELEMENTWISE || call == STENCIL_CALL_APPLY_STENCIL) {
    for (int r = 16; r <= 256; r *= 2) c.push_back({r, 0});
  } else {
    for (int d = 1; d <= 2; ++d)
      for (int r = 64; r <= 1024; r *= 2) c.push_back({r, d});
  }
  return c;
}

}  // namespace

Tuning tuning_lookup(int call, const Geo &q) {
  std::call_once(g_env_once, load_env_cache);
  Tuning t;
  if (g_count.load(std::memory_order_acquire) == 0) return t;
  Entry e;
  if (get(make_key(device_name(), call, q), e)) {
    t.chunk = e.chunk;
    t.depth = e.depth;
  }
  return t;
}


// Times one call of `call` on the scratch arrays (stream-ordered, CUDA events).
static int time_call(const stencil_grid_t *g, int call, int sweeps, double *u, double *f, double *y, void *ws,
                     size_t wsb, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float *ms) {
  int rc = STENCIL_OK;
  cudaEventRecord(e0, s);
  switch (call) {
    case STENCIL_CALL_APPLY_ELEMENTWISE: rc = stencil_apply(g, u, y, STENCIL_FORM_ELEMENTWISE, s); break;
    case STENCIL_CALL_APPLY_STENCIL: rc = stencil_apply(g, u, y, STENCIL_FORM_STENCIL, s); break;
    case STENCIL_CALL_SMOOTH_COLOURED: rc = stencil_smooth_coloured(g, u, f, sweeps, ws, wsb, s); break;
    default: rc = stencil_smooth_jacobi(g, u, f, y, sweeps, 2.0 / 3.0, ws, wsb, s); break;
  }
  cudaEventRecord(e1, s);
  if (rc) return rc;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
    return set_error(STENCIL_ECUDA, "autotune: timing failed");
  return STENCIL_OK;
}

}  // namespace stencil

using namespace stencil;

extern "C" {

int stencil_autotune(const stencil_grid_t *g, int call, int sweeps, stencil_tuning_t *out, void *stream) {
  int rc = check_grid(g);
  if (rc) return rc;
  if (!out) return set_error(STENCIL_EINVAL, "autotune: out is NULL");
  if (!tunable_call(call)) return set_error(STENCIL_EINVAL, "autotune: call cannot be tuned");
  if (g->dtype != STENCIL_F64 || g->op != STENCIL_OP_Q1)
    return set_error(STENCIL_EINVAL, "autotune: F64 and the Q1 operator only");
  const bool smoother = call == STENCIL_CALL_SMOOTH_COLOURED || call == STENCIL_CALL_SMOOTH_JACOBI;
  if (smoother && (sweeps < 2 || sweeps > 1000))
    return set_error(STENCIL_EINVAL, "autotune: smoothers are tuned for 2 to 1000 sweeps per call");
  const Geo q = make_geo(*g);
  cudaStream_t s = (cudaStream_t)stream;
  size_t wsb = 0;
  if (smoother && (rc = stencil_workspace_size(g, call, sweeps, &wsb))) return rc;
  const size_t bytes = (size_t)span_elems(q) * sizeof(double);
  double *u = nullptr, *f = nullptr, *y = nullptr;
  void *ws = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    cudaStreamSynchronize(s);
    cudaFree(u);
    cudaFree(f);
    cudaFree(y);
    cudaFree(ws);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaMalloc(&u, bytes) || cudaMalloc(&f, bytes) || cudaMalloc(&y, bytes) ||
      (wsb && cudaMalloc(&ws, wsb)) || cudaEventCreate(&e0) || cudaEventCreate(&e1)) {
    cudaGetLastError();
    cleanup();
    return set_error(STENCIL_ENOMEM, "autotune: scratch allocation failed");
  }
  const int dim = g->dim;
  const unsigned nb = (unsigned)(4 * device_sm_count());
  k_tune_fill<<<nb, 256, 0, s>>>(u, q, dim, 11);
  k_tune_fill<<<nb, 256, 0, s>>>(f, q, dim, 12);
  k_tune_fill<<<nb, 256, 0, s>>>(y, q, dim, 13);
  if (cudaGetLastError() != cudaSuccess) {
    cleanup();
    return set_error(STENCIL_ECUDA, "autotune: fill failed");
  }
  const Key key = make_key(device_name(), call, q);
  Entry prior;
  const bool had = get(key, prior);
  Entry best;
  best.ms = 1e30;
  for (const Candidate &c : candidates(call, dim)) {
    Entry e;
    e.chunk = c.chunk;
    e.depth = c.depth;
    put(key, e);
    float ms = 0.0f, t = 0.0f;
    // one untimed call, then the best of three
    rc = time_call(g, call, sweeps, u, f, y, ws, wsb, s, e0, e1, &t);
    for (int r = 0; r < 3 && !rc; ++r) {
      rc = time_call(g, call, sweeps, u, f, y, ws, wsb, s, e0, e1, &t);
      if (!rc && (r == 0 || t < ms)) ms = t;
    }
    if (rc) break;
    if (ms < best.ms) {
      best = e;
      best.ms = ms;
    }
  }
  if (rc) {
    if (had) put(key, prior);
    else erase(key);
    cleanup();
    return rc;
  }
  put(key, best);
  cleanup();
  out->chunk = best.chunk;
  out->depth = best.depth;
  out->ms = best.ms;
  return STENCIL_OK;
}

int stencil_tuning_set(const stencil_grid_t *g, int call, const stencil_tuning_t *t) {
  int rc = check_grid(g);
  if (rc) return rc;
  if (!tunable_call(call)) return set_error(STENCIL_EINVAL, "tuning_set: call cannot be tuned");
  const Key key = make_key(device_name(), call, make_geo(*g));
  if (!t) {
    erase(key);
    return STENCIL_OK;
  }
  if (t->chunk < 0 || t->chunk > 4096 || t->depth < 0 || t->depth > 2)
    return set_error(STENCIL_EINVAL, "tuning_set: need 0 <= chunk <= 4096 and 0 <= depth <= 2");
  Entry e;
  e.chunk = t->chunk;
  e.depth = t->depth;
  e.ms = t->ms;
  put(key, e);
  return STENCIL_OK;
}

int stencil_tuning_get(const stencil_grid_t *g, int call, stencil_tuning_t *t) {
  int rc = check_grid(g);
  if (rc) return rc;
  if (!t) return set_error(STENCIL_EINVAL, "tuning_get: out is NULL");
  if (!tunable_call(call)) return set_error(STENCIL_EINVAL, "tuning_get: call cannot be tuned");
  std::call_once(g_env_once, load_env_cache);
  Entry e;
  if (!get(make_key(device_name(), call, make_geo(*g)), e)) return set_error(STENCIL_ENOTFOUND, "tuning_get: no entry");
  t->chunk = e.chunk;
  t->depth = e.depth;
  t->ms = e.ms;
  return STENCIL_OK;
}

int stencil_tuning_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_table.clear();
  g_count.store(0, std::memory_order_release);
  return STENCIL_OK;
}

int stencil_tuning_save(const char *path) {
  if (!path || !*path) return set_error(STENCIL_EINVAL, "tuning_save: path is empty");
  return save_table(path);
}

int stencil_tuning_load(const char *path) {
  if (!path || !*path) return set_error(STENCIL_EINVAL, "tuning_load: path is empty");
  std::call_once(g_env_once, load_env_cache);
  return load_table(path);
}

}  // extern "C"
