// Batched discovery over many scenes (C-ABI emrt_batch_*): persistent
// traversal launches serve the rays of every scene -- depth-first (one launch
// carrying every chain to its end, the default) or breadth-first (one launch
// per bounce) -- followed by one deduplication, one acceptance and a
// per-scene scatter.  The launch sequence has fixed grids and device-resident
// counts; it is captured once into a CUDA graph and replayed.  The traversal
// variant (form and block size; rays fetched per warp and the ray coherence
// sort for the breadth-first form) is chosen by an autotuner that times every
// candidate on the batch and keeps its choice in a JSON cache file.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "scene.cuh"

struct emrt_batch_s {
  uint32_t n = 0, Kmax = 0;
  std::vector<emrt_scene> scenes;
  std::vector<emrt_trace_params> params;
  std::vector<emrt_paths> outs;
  std::vector<uint32_t> count, n_tx;
  uint64_t total = 0;  // primary items over all scenes
  BatchScene *h_tab = nullptr, *d_tab = nullptr;
  std::vector<float4 *> dirs;  // per scene (shared when the ray sets match)
  std::vector<float4 *> owned_dirs;
  Ray *rays[2] = {nullptr, nullptr};
  KeyW<1> *rkeys[2] = {nullptr, nullptr};
  uint32_t *rvals[2] = {nullptr, nullptr};
  uint32_t cand_cap = 0, want_cand = 0;
  uint32_t *cand = nullptr, *uniq = nullptr, *head = nullptr, *pos = nullptr;
  float4 *apts = nullptr;  // acceptance scratch (reflection points)
  KeyW<4> *keys[2] = {nullptr, nullptr};
  uint32_t *vals[2] = {nullptr, nullptr};
  uint32_t *first = nullptr, *cnt = nullptr;
  Counters *ctr = nullptr;
  uint32_t *hist = nullptr, *partial = nullptr;
  KeyLayout kl{};
  int variant = default_bounce_variant();
  bool sort_rays = false;
  uint32_t largest = 0;  // scene whose box quantises the ray sort keys
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream the graph is captured on
  std::string tune_key;
};

namespace {

emrt_status st_of(cudaError_t e) {
  if (e == cudaSuccess) return EMRT_OK;
  if (e == cudaErrorMemoryAllocation) return EMRT_ERR_OOM;
  return EMRT_ERR_CUDA;
}
#define BCK(x)                                  \
  do {                                          \
    cudaError_t _e = (x);                       \
    if (_e != cudaSuccess) return st_of(_e);    \
  } while (0)

void free_scratch(emrt_batch_s *b) {
  cudaFree(b->cand); cudaFree(b->uniq); cudaFree(b->head); cudaFree(b->pos); cudaFree(b->apts);
  for (int k = 0; k < 2; k++) { cudaFree(b->keys[k]); cudaFree(b->vals[k]); }
  b->cand = b->uniq = b->head = b->pos = nullptr;
  b->apts = nullptr;
  b->keys[0] = b->keys[1] = nullptr;
  b->vals[0] = b->vals[1] = nullptr;
  b->cand_cap = 0;
}

cudaError_t alloc_cand(emrt_batch_s *b, uint64_t cap) {
  free_scratch(b);
  cap = std::max<uint64_t>(cap, 1024);
  cudaError_t e;
  if ((e = cudaMalloc(&b->cand, 32 * cap))) return e;
  if ((e = cudaMalloc(&b->uniq, 32 * cap))) return e;
  if ((e = cudaMalloc(&b->head, 4 * cap))) return e;
  if ((e = cudaMalloc(&b->pos, 4 * cap))) return e;
  if ((e = cudaMalloc(&b->apts, sizeof(float4) * (EMRT_MAX_DEPTH + 2) * cap))) return e;
  for (int k = 0; k < 2; k++) {
    if ((e = cudaMalloc(&b->keys[k], sizeof(KeyW<4>) * cap))) return e;
    if ((e = cudaMalloc(&b->vals[k], 4 * cap))) return e;
  }
  b->cand_cap = (uint32_t)cap;
  return cudaSuccess;
}

// ray buffers and sort scratch of the breadth-first variants (the
// depth-first ones keep their rays in registers)
void free_rays(emrt_batch_s *b) {
  for (int k = 0; k < 2; k++) {
    cudaFree(b->rays[k]);
    cudaFree(b->rkeys[k]);
    cudaFree(b->rvals[k]);
    b->rays[k] = nullptr;
    b->rkeys[k] = nullptr;
    b->rvals[k] = nullptr;
  }
}

cudaError_t alloc_rays(emrt_batch_s *b) {
  if (b->Kmax == 0 || b->rays[0]) return cudaSuccess;
  cudaError_t e;
  for (int k = 0; k < 2; k++) {
    if ((e = cudaMalloc(&b->rays[k], sizeof(Ray) * b->total))) return e;
    if ((e = cudaMalloc(&b->rkeys[k], sizeof(KeyW<1>) * b->total))) return e;
    if ((e = cudaMalloc(&b->rvals[k], sizeof(uint32_t) * b->total))) return e;
  }
  return cudaSuccess;
}

void drop_graph(emrt_batch_s *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// current per-scene table (host side, pinned)
void fill_table(emrt_batch_s *b) {
  uint32_t begin = 0;
  for (uint32_t i = 0; i < b->n; i++) {
    emrt_scene s = b->scenes[i];
    BatchScene &t = b->h_tab[i];
    t.g = emrt::geom(s);
    t.dirs = b->dirs[i];
    t.count = b->count[i];
    t.prim_begin = begin;
    t.n_primary = b->count[i] * b->n_tx[i];
    begin += t.n_primary;
    t.K = b->params[i].max_depth;
    t.kappa = (float)(1.25 * sqrt(8.0 * 3.14159265358979323846 /
                                  (3.0 * sqrt(3.0) * (double)b->params[i].n_rays)));
    t.out_rec = b->outs[i].rec;
    t.out_cap = b->outs[i].capacity;
    t.out_count = b->outs[i].count;
  }
}

// the whole launch sequence of one batched trace (capturable)
void enqueue(emrt_batch_s *b, int variant, bool sort_rays, cudaStream_t st) {
  Counters *c = b->ctr;
  cudaMemsetAsync(reinterpret_cast<char *>(c) + sizeof(uint32_t), 0,
                  sizeof(Counters) - sizeof(uint32_t), st);
  const bool walk = bounce_variant_depth_first(variant);
  for (uint32_t bb = 0; bb <= (walk ? 0u : b->Kmax); bb++) {
    BounceLaunch L{};
    L.rin = bb ? b->rays[(bb - 1) & 1] : nullptr;
    L.order = nullptr;
    if (bb > 0 && sort_rays && !walk) {
      launch_ray_keys(L.rin, &c->n_ray[bb], b->scenes[b->largest]->bbox, b->rkeys[0], b->rvals[0],
                      st, true);
      bool alt = radix_sort<1>(&c->n_ray[bb], b->rkeys[0], b->rvals[0], b->rkeys[1], b->rvals[1], 24,
                               b->hist, st, b->total);
      L.order = b->rvals[alt ? 1 : 0];
    }
    L.n_in = &c->n_ray[bb];
    L.n_primary = (uint32_t)b->total;
    L.dirs = nullptr;
    L.count = 0;
    L.rout = b->rays[bb & 1];
    L.n_out = &c->n_ray[bb + 1];
    L.cand = b->cand;
    L.cand_cap = b->cand_cap;
    L.n_cand = &c->n_cand;
    L.work = &c->work[bb];
    L.ctr = c;
    L.kappa = 0.f;
    L.b = (int)bb;
    L.K = (int)b->Kmax;
    launch_bounce_batched(variant, L, b->d_tab, b->n, st);
  }
  // deduplicate (keys carry the scene), accept, scatter to each scene
  launch_path_keys(b->cand, &c->n_cand, b->cand_cap, b->kl, b->keys[0], b->vals[0], &c->n_eff, st);
  const int passes = (b->kl.total + 7) / 8;
  const int first = passes > kDedupPasses + 1 ? passes - kDedupPasses : 0;
  bool alt = radix_sort<4>(&c->n_eff, b->keys[0], b->vals[0], b->keys[1], b->vals[1], b->kl.total,
                           b->hist, st, b->cand_cap, first);
  KeyW<4> *ks = b->keys[alt ? 1 : 0];
  uint32_t *vs = b->vals[alt ? 1 : 0];
  if (first) launch_sort_runs(ks, vs, &c->n_eff, 8 * first, st);
  launch_heads(ks, &c->n_eff, b->head, st);
  exclusive_scan(&c->n_eff, b->head, b->pos, &c->n_unique, b->partial, st);
  launch_unique(b->cand, ks, vs, b->head, b->pos, &c->n_eff, b->uniq, st);
  launch_accept_batched(b->d_tab, b->uniq, &c->n_unique, c, b->apts, b->cand_cap, st);
  launch_keep_flags(b->uniq, &c->n_unique, 0, b->head, st);
  exclusive_scan(&c->n_unique, b->head, b->pos, &c->n_accepted, b->partial, st);
  launch_batch_scatter(b->d_tab, b->n, b->uniq, &c->n_unique, b->head, b->pos, b->first, b->cnt,
                       c, st);
}

// ---------------------------------------------------------------------------
// autotune cache: a flat JSON object {"key": "variant,sort", ...}
std::mutex g_tune_mu;

std::string tune_path() {
  const char *p = getenv("EMRT_AUTOTUNE_CACHE");
  if (p && *p) return p;
  const char *h = getenv("HOME");
  return std::string(h && *h ? h : "/tmp") + "/.emrt_autotune.json";
}

std::map<std::string, std::string> tune_load() {
  std::map<std::string, std::string> m;
  std::ifstream f(tune_path());
  if (!f) return m;
  std::stringstream ss;
  ss << f.rdbuf();
  std::string s = ss.str();
  size_t i = 0;
  auto str = [&](std::string &out) {
    size_t a = s.find('"', i);
    if (a == std::string::npos) return false;
    size_t z = s.find('"', a + 1);
    if (z == std::string::npos) return false;
    out = s.substr(a + 1, z - a - 1);
    i = z + 1;
    return true;
  };
  std::string k, v;
  while (str(k) && str(v)) m[k] = v;
  return m;
}

void tune_store(const std::string &key, const std::string &val) {
  auto m = tune_load();
  m[key] = val;
  std::ofstream f(tune_path());
  if (!f) return;
  f << "{\n";
  size_t i = 0;
  for (auto &kv : m) f << "  \"" << kv.first << "\": \"" << kv.second << "\"" << (++i < m.size() ? ",\n" : "\n");
  f << "}\n";
}

}  // namespace

extern "C" {

emrt_status emrt_batch_create(const emrt_scene *scenes, uint32_t n, const emrt_trace_params *params,
                              emrt_paths *outs, uint32_t flags, emrt_stream stream,
                              emrt_batch *out) {
  if (!scenes || !params || !outs || !out || n == 0 || n > kBatchMaxScenes)
    return EMRT_ERR_INVALID_ARG;
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  emrt_batch_s *b = new emrt_batch_s();
  auto fail = [&](emrt_status e) {
    emrt_batch_destroy(b);
    return e;
  };
  b->n = n;
  uint32_t max_rx = 1, max_tx = 1, max_f = 1;
  uint64_t tris = 0;
  for (uint32_t i = 0; i < n; i++) {
    emrt_scene s = scenes[i];
    const emrt_trace_params &p = params[i];
    if (!s || !s->updated) return fail(EMRT_ERR_STATE);
    if (!outs[i].rec || !outs[i].count || p.max_depth > EMRT_MAX_DEPTH || p.n_rays == 0 ||
        p.ray_stride == 0 || p.ray_offset >= p.n_rays || s->n_tx > kBatchMaxTx)
      return fail(EMRT_ERR_INVALID_ARG);
    uint64_t count = p.ray_count ? p.ray_count
                                 : (p.n_rays - p.ray_offset + p.ray_stride - 1) / p.ray_stride;
    if (count == 0 || count > kBatchMaxCount ||
        p.ray_offset + (count - 1) * p.ray_stride >= p.n_rays)
      return fail(EMRT_ERR_INVALID_ARG);
    b->scenes.push_back(s);
    b->params.push_back(p);
    b->outs.push_back(outs[i]);
    b->count.push_back((uint32_t)count);
    b->n_tx.push_back(s->n_tx);
    b->total += count * s->n_tx;
    b->Kmax = std::max(b->Kmax, p.max_depth);
    max_rx = std::max(max_rx, s->max_rx);
    max_tx = std::max(max_tx, s->n_tx);
    max_f = std::max(max_f, s->Fs + 6 * s->V + 1);
    if (s->T > b->scenes[b->largest]->T) b->largest = i;
    tris += s->T;
  }
  if (b->total >= (1ull << 32)) return fail(EMRT_ERR_INVALID_ARG);
  b->kl = key_layout(max_tx, max_rx, max_f, (int)b->Kmax, n);
  if (b->kl.total > 128) return fail(EMRT_ERR_INVALID_ARG);
  BCK(cudaMallocHost(&b->h_tab, sizeof(BatchScene) * n));
  BCK(cudaMalloc(&b->d_tab, sizeof(BatchScene) * n));
  BCK(cudaMalloc(&b->ctr, sizeof(Counters)));
  BCK(cudaMalloc(&b->hist, sizeof(uint32_t) * (256 * kPrimGrid + 1)));
  BCK(cudaMalloc(&b->partial, sizeof(uint32_t) * (kPrimGrid + 1)));
  BCK(cudaMalloc(&b->first, sizeof(uint32_t) * kBatchMaxScenes));
  BCK(cudaMalloc(&b->cnt, sizeof(uint32_t) * kBatchMaxScenes));
  BCK(cudaMemsetAsync(b->ctr, 0, sizeof(Counters), st));
  // direction tables, shared between scenes with the same ray set
  KeyW<1> *k0 = nullptr;
  uint32_t *v0 = nullptr;
  uint32_t cmax = *std::max_element(b->count.begin(), b->count.end());
  BCK(cudaMalloc(&k0, sizeof(KeyW<1>) * 2 * cmax));
  BCK(cudaMalloc(&v0, sizeof(uint32_t) * 2 * cmax));
  for (uint32_t i = 0; i < n; i++) {
    float4 *found = nullptr;
    for (uint32_t j = 0; j < i; j++)
      if (params[j].n_rays == params[i].n_rays && params[j].ray_offset == params[i].ray_offset &&
          params[j].ray_stride == params[i].ray_stride && b->count[j] == b->count[i])
        found = b->dirs[j];
    if (!found) {
      cudaError_t e = cudaMalloc(&found, sizeof(float4) * b->count[i]);
      if (e) { cudaFree(k0); cudaFree(v0); return fail(st_of(e)); }
      b->owned_dirs.push_back(found);
      build_dir_table(params[i].n_rays, params[i].ray_offset, params[i].ray_stride, b->count[i],
                      found, k0, k0 + b->count[i], v0, v0 + b->count[i], &b->ctr->tmp, b->hist, st);
    }
    b->dirs.push_back(found);
  }
  cudaStreamSynchronize(st);
  cudaFree(k0);
  cudaFree(v0);
  uint64_t want = 0;
  for (uint32_t i = 0; i < n; i++)
    want += 4ull * b->scenes[i]->n_tx * b->scenes[i]->n_rx * (b->params[i].max_depth + 1);
  BCK(alloc_cand(b, std::max<uint64_t>(want, 1u << 16)));
  // autotune (or read the cached choice)
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, dev);
  char key[512];
  snprintf(key, sizeof(key), "%.256s|scenes=%u|rays=%llu|tris=%llu|K=%u", prop.name, n,
           (unsigned long long)b->total, (unsigned long long)tris, b->Kmax);
  b->tune_key = key;
  fill_table(b);
  BCK(cudaMemcpyAsync(b->d_tab, b->h_tab, sizeof(BatchScene) * n, cudaMemcpyHostToDevice, st));
  std::string cached;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto m = tune_load();
    auto it = m.find(b->tune_key);
    if (it != m.end()) cached = it->second;
  }
  if (!cached.empty()) {
    int v = 1, so = 1;
    if (sscanf(cached.c_str(), "%d,%d", &v, &so) == 2 && v >= 0 && v < n_bounce_variants()) {
      b->variant = v;
      b->sort_rays = so != 0;
    }
  } else if (flags & EMRT_BATCH_AUTOTUNE) {
    BCK(alloc_rays(b));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int so = 0; so < 2; so++) {
      for (int v = 0; v < n_bounce_variants(); v++) {
        if (so && bounce_variant_depth_first(v)) continue;  // no ray sort to switch
        for (int rep = 0; rep < 2; rep++) {  // first run warms caches, second is timed
          cudaEventRecord(e0, st);
          enqueue(b, v, so != 0, st);
          cudaEventRecord(e1, st);
          cudaEventSynchronize(e1);
        }
        Counters h;
        cudaMemcpy(&h, b->ctr, sizeof(Counters), cudaMemcpyDeviceToHost);
        if (h.n_cand > b->cand_cap) {  // grow and retry this variant
          BCK(alloc_cand(b, (uint64_t)h.n_cand + h.n_cand / 4 + 1024));
          v--;
          cudaMemset(b->ctr, 0, sizeof(uint32_t));
          continue;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        bool ok = (h.err & ERR_STACK) == 0;
        cudaMemset(b->ctr, 0, sizeof(uint32_t));
        if (ok && ms < best) {
          best = ms;
          b->variant = v;
          b->sort_rays = so != 0;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    char val[64];
    snprintf(val, sizeof(val), "%d,%d", b->variant, b->sort_rays ? 1 : 0);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_store(b->tune_key, val);
  } else if (flags & EMRT_BATCH_BREADTH_FIRST) {
    b->variant = default_breadth_first_variant();
    b->sort_rays = true;
  }
  if (bounce_variant_depth_first(b->variant)) {
    cudaStreamSynchronize(st);
    free_rays(b);
  } else {
    BCK(alloc_rays(b));
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (!e) e = cudaGetLastError();
  if (e) return fail(st_of(e));
  *out = b;
  return EMRT_OK;
}

}  // extern "C"

namespace {
// batches of emrt_trace_batched, keyed by the bytes of their argument arrays
std::mutex g_reg_mu;
std::map<std::string, emrt_batch> g_reg;
std::string batch_key(const emrt_scene *scenes, uint32_t n, const emrt_trace_params *params,
                      const emrt_paths *outs) {
  std::string k;
  auto put = [&](uint64_t v) { k.append(reinterpret_cast<const char *>(&v), sizeof(v)); };
  for (uint32_t i = 0; i < n; i++) {  // field by field: struct padding is not part of it
    put((uint64_t)(uintptr_t)scenes[i]);
    const emrt_trace_params &p = params[i];
    put(p.max_depth);
    put(p.n_rays);
    put(p.ray_offset);
    put(p.ray_stride);
    put(p.ray_count);
    put(p.flags);
    put((uint64_t)(uintptr_t)outs[i].rec);
    put(outs[i].capacity);
    put((uint64_t)(uintptr_t)outs[i].count);
  }
  return k;
}
}  // namespace

// Drops the registered batches that use scene s (called by emrt_scene_destroy).
void batch_forget_scene(emrt_scene s) {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  for (auto it = g_reg.begin(); it != g_reg.end();) {
    bool uses = false;
    for (emrt_scene q : it->second->scenes) uses |= q == s;
    if (uses) {
      emrt_batch_destroy(it->second);
      it = g_reg.erase(it);
    } else {
      ++it;
    }
  }
}

extern "C" {

emrt_status emrt_trace_batched(const emrt_scene *scenes, uint32_t n,
                               const emrt_trace_params *params, emrt_paths *outs,
                               emrt_stream s) {
  if (!scenes || !params || !outs || n == 0 || n > kBatchMaxScenes) return EMRT_ERR_INVALID_ARG;
  emrt_batch b = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_reg_mu);
    const std::string key = batch_key(scenes, n, params, outs);
    auto it = g_reg.find(key);
    if (it != g_reg.end()) {
      b = it->second;
    } else {
      emrt_status e = emrt_batch_create(scenes, n, params, outs, 0u, s, &b);
      if (e != EMRT_OK) return e;
      g_reg[key] = b;
    }
  }
  emrt_status e = emrt_batch_trace(b, s);
  if (e != EMRT_OK) return e;
  return emrt_batch_sync(b, s, nullptr);
}

void emrt_batch_destroy(emrt_batch b) {
  if (!b) return;
  drop_graph(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  free_scratch(b);
  free_rays(b);
  for (auto p : b->owned_dirs) cudaFree(p);
  cudaFree(b->d_tab); cudaFree(b->ctr); cudaFree(b->hist); cudaFree(b->partial);
  cudaFree(b->first); cudaFree(b->cnt);
  if (b->h_tab) cudaFreeHost(b->h_tab);
  delete b;
}

emrt_status emrt_batch_trace(emrt_batch b, emrt_stream stream) {
  if (!b) return EMRT_ERR_INVALID_ARG;
  for (uint32_t i = 0; i < b->n; i++)
    if (b->scenes[i]->n_tx != b->n_tx[i] || !b->scenes[i]->updated) return EMRT_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  BCK(cudaStreamIsCapturing(st, &cap));
  if (cap == cudaStreamCaptureStatusActive) {
    // the caller is capturing its own graph: record the table copy and the
    // batch's launch sequence into it (no host sync, no allocation; the
    // batch must have been traced once before, so that its scratch is sized)
    if (!b->exec) return EMRT_ERR_STATE;
    fill_table(b);
    BCK(cudaMemcpyAsync(b->d_tab, b->h_tab, sizeof(BatchScene) * b->n, cudaMemcpyHostToDevice, st));
    enqueue(b, b->variant, b->sort_rays, st);
    return EMRT_OK;
  }
  if (b->want_cand > b->cand_cap) {  // a previous call overflowed: grow, re-capture
    drop_graph(b);
    BCK(alloc_cand(b, b->want_cand));
  }
  BCK(cudaStreamSynchronize(st));  // the pinned table may still be read by a copy
  fill_table(b);
  BCK(cudaMemcpyAsync(b->d_tab, b->h_tab, sizeof(BatchScene) * b->n, cudaMemcpyHostToDevice, st));
  if (!b->exec) {
    // capture on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured); the graph is launched on the
    // caller's stream below
    if (!b->cap_stream) BCK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    bounce_variant_grid(b->variant);  // occupancy query before the capture starts
    BCK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    enqueue(b, b->variant, b->sort_rays, b->cap_stream);
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &b->graph);
    if (e) { drop_graph(b); return st_of(e); }
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e) { drop_graph(b); return st_of(e); }
  }
  BCK(cudaGraphLaunch(b->exec, st));
  return EMRT_OK;
}

emrt_status emrt_batch_sync(emrt_batch b, emrt_stream stream, emrt_stats *out) {
  if (!b) return EMRT_ERR_INVALID_ARG;
  BCK(cudaStreamSynchronize((cudaStream_t)stream));
  Counters h;
  BCK(cudaMemcpy(&h, b->ctr, sizeof(Counters), cudaMemcpyDeviceToHost));
  BCK(cudaMemset(b->ctr, 0, sizeof(uint32_t)));
  if (h.n_cand > b->cand_cap)
    b->want_cand = (uint32_t)std::min<uint64_t>((uint64_t)h.n_cand + h.n_cand / 4 + 1024, 0x7fffffffull);
  if (out) {
    memset(out, 0, sizeof(*out));
    for (int k = 0; k <= EMRT_MAX_DEPTH; k++) out->segments[k] = h.segments[k];
    out->candidates = h.n_cand;
    out->unique_candidates = h.n_unique;
    out->accepted = h.n_accepted;
    out->occlusion_rays = h.occl_rays;
    out->node_visits = h.node_visits;
    out->tri_tests = h.tri_tests;
    out->dyn_node_visits = h.dyn_node_visits;
    out->box_tests = h.box_tests;
    out->rx_node_visits = h.rx_node_visits;
    out->rx_tests = h.rx_tests;
    out->error_bits = h.err;
    out->required_candidates = h.n_cand;
    out->required_paths = h.n_accepted;
  }
  if (h.err & ERR_STACK) return EMRT_ERR_DEVICE;
  if (h.err & (ERR_CAND_OVERFLOW | ERR_PATH_OVERFLOW | ERR_RAY_OVERFLOW) || h.n_cand > b->cand_cap)
    return EMRT_ERR_CAPACITY;
  return EMRT_OK;
}

emrt_status emrt_batch_config(emrt_batch b, char *buf, uint32_t len) {
  if (!b || !buf || len == 0) return EMRT_ERR_INVALID_ARG;
  snprintf(buf, len, "%s sort=%d", bounce_variant_name(b->variant), b->sort_rays ? 1 : 0);
  return EMRT_OK;
}

}  // extern "C"
