// C-ABI of libemrt.so: scene lifetime, argument checks, scratch management
// and the order of kernel launches for each entry point.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "bvh.cuh"
#include "field.cuh"
#include "trace.cuh"
#include "scene.cuh"

using namespace emrt;

namespace emrt {
static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(); }
}  // namespace emrt

namespace {

emrt_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return EMRT_OK;
  if (e == cudaErrorMemoryAllocation) return EMRT_ERR_OOM;
  return EMRT_ERR_CUDA;
}

#define CK(x)                                   \
  do {                                          \
    cudaError_t _e = (x);                       \
    if (_e != cudaSuccess) return cuda_status(_e); \
  } while (0)

template <typename T>
cudaError_t grow(T **p, uint64_t &cap, uint64_t need) {
  if (need <= cap && *p) return cudaSuccess;
  cudaFree(*p);
  *p = nullptr;
  cap = 0;
  cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (need ? need : 1));
  if (e == cudaSuccess) cap = need;
  return e;
}

__global__ void k_faces(const uint32_t *off, const float *xyz, const uint32_t *mat, uint32_t F,
                        double4_32a *plane, uint4 *info, float4 *vert) {
  uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  uint32_t a = off[f], nv = off[f + 1] - off[f];
  double nx = 0, ny = 0, nz = 0, cx = 0, cy = 0, cz = 0;
  for (uint32_t i = 0; i < nv; i++) {
    const float *p = xyz + 3ull * (a + i);
    const float *q = xyz + 3ull * (a + (i + 1) % nv);
    double px = p[0], py = p[1], pz = p[2], qx = q[0], qy = q[1], qz = q[2];
    // Newell's normal of a planar polygon
    nx += (py - qy) * (pz + qz);
    ny += (pz - qz) * (px + qx);
    nz += (px - qx) * (py + qy);
    cx += px; cy += py; cz += pz;
    vert[a + i] = make_float4(p[0], p[1], p[2], 0.f);
  }
  double l = sqrt(nx * nx + ny * ny + nz * nz);
  nx /= l; ny /= l; nz /= l;
  plane[f] = make_double4_32a(nx, ny, nz, (nx * cx + ny * cy + nz * cz) / nv);
  info[f] = make_uint4(a, nv, mat[f], 0u);
}

__global__ void k_half(const float *h, uint32_t V, float4 *out) {
  uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < V) out[v] = make_float4(h[3 * v], h[3 * v + 1], h[3 * v + 2], 0.f);
}

// per-frame state: box corners in float32 arithmetic, receivers, transmitters
__global__ void k_update(const float *vp, const float *vv, const float4 *half, uint32_t V,
                         float4 *lo, float4 *hi, float4 *vel, const float *rp, const float *rv,
                         uint32_t R, float4 *rxp, float4 *rxv, const float *tp, const float *tv,
                         uint32_t X, float4 *txp, float4 *txv) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < V) {
    float4 h = half[i];
    float x = vp[3 * i], y = vp[3 * i + 1], z = vp[3 * i + 2];
    lo[i] = make_float4(__fsub_rn(x, h.x), __fsub_rn(y, h.y), __fsub_rn(z, h.z), 0.f);
    hi[i] = make_float4(__fadd_rn(x, h.x), __fadd_rn(y, h.y), __fadd_rn(z, h.z), 0.f);
    vel[i] = vv ? make_float4(vv[3 * i], vv[3 * i + 1], vv[3 * i + 2], 0.f) : make_float4(0, 0, 0, 0);
  }
  if (i < R) {
    rxp[i] = make_float4(rp[3 * i], rp[3 * i + 1], rp[3 * i + 2], 0.f);
    rxv[i] = rv ? make_float4(rv[3 * i], rv[3 * i + 1], rv[3 * i + 2], 0.f) : make_float4(0, 0, 0, 0);
  }
  if (i < X) {
    txp[i] = make_float4(tp[3 * i], tp[3 * i + 1], tp[3 * i + 2], 0.f);
    txv[i] = tv ? make_float4(tv[3 * i], tv[3 * i + 1], tv[3 * i + 2], 0.f) : make_float4(0, 0, 0, 0);
  }
}

// corners of the merged per-frame tree: vehicle boxes, then receiver points
__global__ void k_mix_prims(const float4 *vlo, const float4 *vhi, uint32_t V, const float4 *rx,
                            uint32_t R, float4 *lo, float4 *hi) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < V) {
    lo[i] = vlo[i];
    hi[i] = vhi[i];
  } else if (i < V + R) {
    lo[i] = hi[i] = rx[i - V];
  }
}

__global__ void k_check_cand(Counters *c, uint32_t cap) {
  if (c->n_cand > cap) atomicOr(&c->err, ERR_CAND_OVERFLOW);
}

__global__ void k_publish_count(const Counters *c, uint32_t *count) { *count = c->n_accepted; }

__global__ void k_clamp_count(const uint32_t *n, uint32_t cap, uint32_t *out) { *out = min(*n, cap); }

// records removed by the last revalidation: entered - kept
__global__ void k_evicted(const Counters *c, uint32_t *out) { *out = c->n_eff - c->n_accepted; }
void launch_evicted(const Counters *c, uint32_t *out, cudaStream_t s) {
  emrt::note_launch(), k_evicted<<<1, 1, 0, s>>>(c, out);
}

cudaError_t ensure_cand(emrt_scene_s *s, uint64_t need) {
  if (need <= s->cand_cap && s->cand) return cudaSuccess;
  uint64_t c = 0;
  cudaError_t e;
  uint64_t cap = std::max<uint64_t>(need, 1024);
  if (cap > 0xffffffffull / 2) cap = 0xffffffffull / 2;
  e = grow(&s->cand, c, cap * 8); if (e) return e; c = 0;
  e = grow(&s->uniq, c, cap * 8); if (e) return e; c = 0;
  e = grow(&s->head, c, cap); if (e) return e; c = 0;
  e = grow(&s->pos, c, cap); if (e) return e; c = 0;
  e = grow(&s->apts, c, cap * (EMRT_MAX_DEPTH + 2)); if (e) return e; c = 0;
  for (int k = 0; k < 2; k++) {
    e = grow(&s->keys[k], c, cap); if (e) return e; c = 0;
    e = grow(&s->vals[k], c, cap); if (e) return e; c = 0;
  }
  s->cand_cap = (uint32_t)cap;
  return cudaSuccess;
}

// Sort + unique of records [0, *n) of `src` (capacity cap) into s->uniq;
// unique count in ctr->n_unique.
void dedup(emrt_scene_s *s, const uint32_t *src, const uint32_t *n, uint32_t cap, KeyLayout kl,
           cudaStream_t st) {
  Counters *c = s->ctr;
  launch_path_keys(src, n, cap, kl, s->keys[0], s->vals[0], &c->n_eff, st);
  // radix passes over the top kDedupPasses bytes only; the runs equal there
  // (a few candidates each) are then sorted in place by the whole key
  const int passes = (kl.total + 7) / 8;
  const int first = passes > kDedupPasses + 1 ? passes - kDedupPasses : 0;
  bool alt = radix_sort<4>(&c->n_eff, s->keys[0], s->vals[0], s->keys[1], s->vals[1], kl.total,
                           s->hist, st, cap, first);
  KeyW<4> *ks = s->keys[alt ? 1 : 0];
  uint32_t *vs = s->vals[alt ? 1 : 0];
  if (first) launch_sort_runs(ks, vs, &c->n_eff, 8 * first, st);
  launch_heads(ks, &c->n_eff, s->head, st);
  exclusive_scan(&c->n_eff, s->head, s->pos, &c->n_unique, s->partial, st);
  launch_unique(src, ks, vs, s->head, s->pos, &c->n_eff, s->uniq, st);
}

emrt_status check_paths(const emrt_paths *p) {
  if (!p || !p->rec || !p->count) return EMRT_ERR_INVALID_ARG;
  return EMRT_OK;
}

}  // namespace

extern "C" {

uint64_t emrt_kernel_launches(void) { return emrt::launch_count(); }

emrt_status emrt_selftest_grid_barrier(uint32_t missing_blocks, uint32_t *blocks_passed,
                                       uint32_t *timed_out) {
  if (!blocks_passed || !timed_out || missing_blocks > 1024u) return EMRT_ERR_INVALID_ARG;
  cudaError_t e = emrt::grid_barrier_selftest(missing_blocks, blocks_passed, timed_out);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return EMRT_ERR_CUDA;
  }
  return EMRT_OK;
}

const char *emrt_status_string(emrt_status e) {
  switch (e) {
    case EMRT_OK: return "ok";
    case EMRT_ERR_INVALID_ARG: return "invalid argument";
    case EMRT_ERR_OOM: return "device allocation failed";
    case EMRT_ERR_CUDA: return "CUDA runtime error";
    case EMRT_ERR_CAPACITY: return "buffer capacity exceeded";
    case EMRT_ERR_TIMEOUT: return "bounded device wait gave up";
    case EMRT_ERR_STATE: return "call order violated";
    case EMRT_ERR_DEVICE: return "kernel-raised error";
  }
  return "unknown status";
}

emrt_status emrt_scene_create(const emrt_scene_desc *d, emrt_stream stream, emrt_scene *out) {
  if (!d || !out) return EMRT_ERR_INVALID_ARG;
  *out = nullptr;
  if ((d->n_static_faces && (!d->face_off || !d->face_xyz || !d->face_mat)) ||
      (d->n_tris && (!d->tri_xyz || !d->tri_face)) || (d->n_vehicles && !d->veh_half) ||
      d->max_tx == 0 || d->max_tx > 255 || d->max_rx == 0)
    return EMRT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  emrt_scene_s *s = new emrt_scene_s();
  cudaGetDevice(&s->device);
  s->Fs = d->n_static_faces;
  s->T = d->n_tris;
  s->V = d->n_vehicles;
  s->max_rx = d->max_rx;
  s->max_tx = d->max_tx;
  s->veh_mat = d->veh_mat;
  s->rebuild_every = d->rebuild_every ? d->rebuild_every : 1;
  auto fail = [&](cudaError_t e) {
    emrt_scene_destroy(s);
    return cuda_status(e);
  };
  cudaError_t e;
  uint64_t c = 0;
  if (s->Fs) {
    e = cudaMemcpy(&s->NV, d->face_off + s->Fs, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e) return fail(e);
  }
  if ((e = grow(&s->face_plane, c, std::max(s->Fs, 1u)))) return fail(e); c = 0;
  if ((e = grow(&s->face_info, c, std::max(s->Fs, 1u)))) return fail(e); c = 0;
  if ((e = grow(&s->face_vert, c, std::max(s->NV, 1u)))) return fail(e); c = 0;
  if ((e = grow(&s->bbox, c, 4))) return fail(e); c = 0;
  if (s->Fs) emrt::note_launch(), k_faces<<<ceil_div(s->Fs, 128), 128, 0, st>>>(d->face_off, d->face_xyz, d->face_mat,
                                                          s->Fs, s->face_plane, s->face_info,
                                                          s->face_vert);
  if ((e = grow(&s->ctr, c, 1))) return fail(e); c = 0;
  if ((e = grow(&s->hist, c, 256 * kPrimGrid + 1))) return fail(e); c = 0;
  for (int k = 0; k < 2; k++) {
    if ((e = grow(&s->hist_side[k], c, 256 * kPrimGrid + 1))) return fail(e); c = 0;
    if ((e = cudaStreamCreateWithFlags(&s->side[k], cudaStreamNonBlocking))) return fail(e);
    if ((e = cudaEventCreateWithFlags(&s->ev_side[k], cudaEventDisableTiming))) return fail(e);
  }
  if ((e = cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming))) return fail(e);
  if ((e = grow(&s->partial, c, kPrimGrid + 1))) return fail(e); c = 0;
  cudaMemsetAsync(s->ctr, 0, sizeof(Counters), st);
  bbox_of_tris(d->tri_xyz, s->T, s->bbox, st);
  // leaf-box pad of every tree of the scene: 2^-21 x the largest static
  // coordinate (at least 1 m), see BVHBuf::pad
  float pad = 4.76837158e-7f;
  if (s->T) {
    float4 bb[2];
    if ((e = cudaMemcpyAsync(bb, s->bbox, sizeof(bb), cudaMemcpyDeviceToHost, st))) return fail(e);
    if ((e = cudaStreamSynchronize(st))) return fail(e);
    float m = 1.f;
    for (float v : {bb[0].x, bb[0].y, bb[0].z, bb[1].x, bb[1].y, bb[1].z})
      if (std::isfinite(v)) m = std::max(m, std::fabs(v));
    pad = 4.76837158e-7f * m;
  }
  if ((e = bvh_alloc(s->stat, PRIM_TRI, std::max(s->T, 2u)))) return fail(e);
  s->stat.pad = pad;
  // static geometry: binned-SAH tree (built once); the LBVH if the SAH tree
  // would be deeper than the traversal stack
  if (bvh_build_tris_sah(s->stat, d->tri_xyz, d->tri_face, s->T, st) != cudaSuccess) {
    cudaGetLastError();
    if ((e = bvh_build_tris(s->stat, d->tri_xyz, d->tri_face, s->T, s->bbox, s->hist, st)))
      return fail(e);
  }
  if ((e = bvh8_build(s->stat, st))) return fail(e);
  if ((e = bvh_alloc(s->dyn, PRIM_BOX, std::max(s->V, 2u)))) return fail(e);
  if ((e = bvh_alloc(s->rxb, PRIM_POINT, std::max(s->max_rx, 2u)))) return fail(e);
  if ((e = bvh_alloc(s->txb, PRIM_POINT, std::max(s->max_tx, 2u)))) return fail(e);
  if ((e = bvh_alloc(s->mix, PRIM_BOX, std::max(s->V + s->max_rx, 2u)))) return fail(e);
  s->dyn.pad = s->rxb.pad = s->txb.pad = s->mix.pad = pad;
  // the per-frame builds report a barrier that gave up through the
  // scene's error word (read by the next emrt_sync)
  s->dyn.err_word = s->rxb.err_word = s->txb.err_word = s->mix.err_word = &s->ctr->err;
  if ((e = grow(&s->mix_lo, c, s->V + s->max_rx))) return fail(e); c = 0;
  if ((e = grow(&s->mix_hi, c, s->V + s->max_rx))) return fail(e); c = 0;
  uint32_t V1 = std::max(s->V, 1u);
  if ((e = grow(&s->veh_half, c, V1))) return fail(e); c = 0;
  if ((e = grow(&s->veh_lo, c, V1))) return fail(e); c = 0;
  if ((e = grow(&s->veh_hi, c, V1))) return fail(e); c = 0;
  if ((e = grow(&s->veh_vel, c, V1))) return fail(e); c = 0;
  if ((e = grow(&s->rx_pos, c, s->max_rx))) return fail(e); c = 0;
  if ((e = grow(&s->rx_vel, c, s->max_rx))) return fail(e); c = 0;
  if ((e = grow(&s->tx_pos, c, s->max_tx))) return fail(e); c = 0;
  if ((e = grow(&s->tx_vel, c, s->max_tx))) return fail(e); c = 0;
  if (s->V) emrt::note_launch(), k_half<<<ceil_div(s->V, 256), 256, 0, st>>>(d->veh_half, s->V, s->veh_half);
  for (int k = 0; k < 4; k++)
    if ((e = cudaEventCreate(&s->ev[k]))) return fail(e);
  for (int k = 0; k < 2 * (EMRT_MAX_DEPTH + 2); k++)
    if ((e = cudaEventCreate(&s->evb[k]))) return fail(e);
  e = cudaStreamSynchronize(st);
  if (!e) e = cudaGetLastError();
  if (e) return fail(e);
  *out = s;
  return EMRT_OK;
}

void emrt_scene_destroy(emrt_scene s) {
  if (!s) return;
  batch_forget_scene(s);
  cudaFree(s->face_plane); cudaFree(s->face_info); cudaFree(s->face_vert); cudaFree(s->bbox);
  bvh_free(s->stat); bvh_free(s->dyn); bvh_free(s->rxb); bvh_free(s->txb); bvh_free(s->mix);
  cudaFree(s->mix_lo); cudaFree(s->mix_hi);
  cudaFree(s->src_pos);
  cudaFree(s->veh_half); cudaFree(s->veh_lo); cudaFree(s->veh_hi); cudaFree(s->veh_vel);
  cudaFree(s->rx_pos); cudaFree(s->rx_vel); cudaFree(s->tx_pos); cudaFree(s->tx_vel);
  cudaFree(s->ctr); cudaFree(s->hist); cudaFree(s->partial);
  for (int k = 0; k < 2; k++) {
    cudaFree(s->hist_side[k]);
    if (s->side[k]) cudaStreamDestroy(s->side[k]);
    if (s->ev_side[k]) cudaEventDestroy(s->ev_side[k]);
  }
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  cudaFree(s->rv_rec); cudaFree(s->rv_head); cudaFree(s->rv_pos); cudaFree(s->rv_partial);
  cudaFree(s->rv_apts); cudaFree(s->rv_ctr);
  for (auto &t : s->dt) {
    cudaFree(t.dirs);
    cudaFree(t.stab);
    cudaFree(t.tx_ref);
    cudaFree(t.tx_epoch);
  }
  cudaFree(s->chain_q);
  cudaFree(s->dt_scratch);
  cudaFree(s->rays[0]); cudaFree(s->rays[1]);
  for (int k = 0; k < 2; k++) { cudaFree(s->rkeys[k]); cudaFree(s->rvals[k]); }
  cudaFree(s->cand); cudaFree(s->uniq); cudaFree(s->head); cudaFree(s->pos); cudaFree(s->apts);
  for (int k = 0; k < 2; k++) { cudaFree(s->keys[k]); cudaFree(s->vals[k]); }
  cudaFree(s->contrib);
  for (int k = 0; k < 4; k++)
    if (s->ev[k]) cudaEventDestroy(s->ev[k]);
  for (int k = 0; k < 2 * (EMRT_MAX_DEPTH + 2); k++)
    if (s->evb[k]) cudaEventDestroy(s->evb[k]);
  delete s;
}

emrt_status emrt_scene_update_dynamic(emrt_scene s, const float *veh_pos, const float *veh_vel,
                                      const float *rx_pos, const float *rx_vel, uint32_t n_rx,
                                      const float *tx_pos, const float *tx_vel, uint32_t n_tx,
                                      emrt_stream stream) {
  if (!s) return EMRT_ERR_INVALID_ARG;
  if ((s->V && !veh_pos) || n_rx == 0 || n_rx > s->max_rx || n_tx == 0 || n_tx > s->max_tx ||
      !rx_pos || !tx_pos)
    return EMRT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  s->n_rx = n_rx;
  s->n_tx = n_tx;
  uint32_t m = std::max(s->V, std::max(n_rx, n_tx));
  emrt::note_launch(), k_update<<<ceil_div(m, 256), 256, 0, st>>>(veh_pos, veh_vel, s->veh_half, s->V, s->veh_lo,
                                             s->veh_hi, s->veh_vel, rx_pos, rx_vel, n_rx,
                                             s->rx_pos, s->rx_vel, tx_pos, tx_vel, n_tx, s->tx_pos,
                                             s->tx_vel);
  // the three per-frame trees are independent small builds (a few tens of
  // blocks per launch): vehicles and receivers on side streams, the merged
  // tree on the caller's stream, joined before the update returns
  CK(cudaEventRecord(s->ev_fork, st));
  for (int k = 0; k < 2; k++) CK(cudaStreamWaitEvent(s->side[k], s->ev_fork, 0));
  if (s->V) {
    if (s->n_updates % s->rebuild_every == 0)
      CK(bvh_build_boxes(s->dyn, s->veh_lo, s->veh_hi, s->V, s->bbox, s->hist_side[0], s->side[0]));
    else
      CK(bvh_refit_boxes(s->dyn, s->veh_lo, s->veh_hi, s->side[0]));
  }
  CK(bvh_build_points(s->rxb, s->rx_pos, n_rx, s->bbox, s->hist_side[1], s->side[1]));
  // vehicles and receivers in one tree for discovery's per-segment query
  const uint32_t nm = s->V + n_rx;
  emrt::note_launch(), k_mix_prims<<<ceil_div(nm, 256), 256, 0, st>>>(s->veh_lo, s->veh_hi, s->V,
                                                                     s->rx_pos, n_rx, s->mix_lo,
                                                                     s->mix_hi);
  CK(bvh_build_boxes(s->mix, s->mix_lo, s->mix_hi, nm, s->bbox, s->hist, st));
  for (int k = 0; k < 2; k++) {
    CK(cudaEventRecord(s->ev_side[k], s->side[k]));
    CK(cudaStreamWaitEvent(st, s->ev_side[k], 0));
  }
  s->n_updates++;
  s->updated = true;
  CK(cudaGetLastError());
  return EMRT_OK;
}

}  // extern "C"

namespace {

// Bits needed to hold 0 .. v-1 (at least 1).
int id_bits(uint64_t v) {
  int b = 1;
  while (b < 32 && (1ull << b) < v) b++;
  return b;
}

// Discovery from the n_src source points gt.tx_pos with reception spheres at
// the points of gt.rxb (forward: transmitters -> receivers; backward:
// receivers -> transmitters), then, when backward, the candidates' reversal
// to forward orientation (receiver ids from rx_ids), and the common tail:
// canonical dedup, image-method acceptance in the scene's forward geometry
// and compaction into out.  count: rays per source; jbits: ray-index bits of
// the ray ids.
// Revalidation of cache on stream st with the scratch (rec, head, pos,
// partial, apts; capacity cap >= cache->capacity) and counters c.
void revalidate_with(emrt_scene_s *s, emrt_paths *cache, uint32_t flags, cudaStream_t st,
                     uint32_t *rec, uint32_t *head, uint32_t *pos, uint32_t *partial,
                     float4 *apts, uint32_t cap, Counters *c) {
  GeomView g = geom(s);
  // clamp the count to the capacity before acceptance
  emrt::note_launch(), k_clamp_count<<<1, 1, 0, st>>>(cache->count, cache->capacity, &c->n_eff);
  launch_copy_records(cache->rec, &c->n_eff, rec, cache->capacity, st);
  launch_accept(g, rec, &c->n_eff, c, apts, cap, st);
  int keep_all = (flags & EMRT_REVALIDATE_KEEP) ? 1 : 0;
  launch_keep_flags(rec, &c->n_eff, keep_all, head, st);
  exclusive_scan(&c->n_eff, head, pos, &c->n_accepted, partial, st);
  launch_scatter(rec, &c->n_eff, head, pos, cache->rec, cache->capacity, &c->n_accepted, c, st);
  emrt::note_launch(), k_publish_count<<<1, 1, 0, st>>>(c, cache->count);
}

// The side-stream revalidation scratch, sized for cap records.
cudaError_t ensure_rv(emrt_scene_s *s, uint64_t cap) {
  if (cap <= s->rv_cap && s->rv_rec) return cudaSuccess;
  cudaFree(s->rv_rec); cudaFree(s->rv_head); cudaFree(s->rv_pos); cudaFree(s->rv_partial);
  cudaFree(s->rv_apts);
  s->rv_rec = s->rv_head = s->rv_pos = s->rv_partial = nullptr;
  s->rv_apts = nullptr;
  s->rv_cap = 0;
  cudaError_t e;
  if ((e = cudaMalloc(&s->rv_rec, sizeof(uint32_t) * 8 * cap))) return e;
  if ((e = cudaMalloc(&s->rv_head, sizeof(uint32_t) * cap))) return e;
  if ((e = cudaMalloc(&s->rv_pos, sizeof(uint32_t) * cap))) return e;
  if ((e = cudaMalloc(&s->rv_partial, sizeof(uint32_t) * (kPrimGrid + 1)))) return e;
  if ((e = cudaMalloc(&s->rv_apts, sizeof(float4) * (EMRT_MAX_DEPTH + 2) * cap))) return e;
  if (!s->rv_ctr && (e = cudaMalloc(&s->rv_ctr, sizeof(Counters)))) return e;
  s->rv_cap = cap;
  return cudaSuccess;
}

// main counters <- error bits and occlusion rays of the side revalidation
__global__ void k_fold_counters(const Counters *side, Counters *c) {
  atomicOr(&c->err, side->err);
  c->occl_rays += side->occl_rays;
}

// Tail of a rediscovery: the unique candidates in s->uniq (count n_unique,
// canonical) that the cache does not hold are accepted, and the accepted
// ones merged into the cache (both canonical and disjoint: a merge-path
// gather, no duplicate runs).
void rediscover_tail(emrt_scene_s *s, const GeomView &g, emrt_paths *cache, cudaStream_t st) {
  Counters *c = s->ctr;
  const KeyLayout kl = key_layout(s->n_tx, s->n_rx, s->Fs + 6 * s->V + 1, EMRT_MAX_DEPTH);
  launch_known(s->uniq, &c->n_unique, cache->rec, cache->count, cache->capacity, kl, s->head, st);
  exclusive_scan(&c->n_unique, s->head, s->pos, &c->n_eff, s->partial, st);
  launch_scatter(s->uniq, &c->n_unique, s->head, s->pos, s->cand, s->cand_cap, &c->n_eff, c, st);
  launch_accept(g, s->cand, &c->n_eff, c, s->apts, s->cand_cap, st);
  launch_keep_flags(s->cand, &c->n_eff, 0, s->head, st);
  exclusive_scan(&c->n_eff, s->head, s->pos, &c->tmp, s->partial, st);
  launch_scatter(s->cand, &c->n_eff, s->head, s->pos, s->uniq, s->cand_cap, &c->tmp, c, st);
  launch_concat(cache->rec, cache->count, cache->capacity, s->uniq, &c->tmp, s->cand_cap, s->cand,
                s->cand_cap, &c->n_accepted, c, st);
  launch_path_keys(s->cand, &c->n_accepted, s->cand_cap, kl, s->keys[0], s->vals[0], &c->n_eff, st);
  launch_merge_path(s->keys[0], s->vals[0], cache->count, cache->capacity, &c->n_eff, s->keys[1],
                    s->vals[1], c, st);
  launch_gather_records(s->cand, s->vals[1], &c->n_eff, cache->rec, cache->capacity, c, st);
  emrt::note_launch(), k_clamp_count<<<1, 1, 0, st>>>(&c->n_eff, 0xffffffffu, cache->count);
}

emrt_status run_trace(emrt_scene_s *s, const emrt_trace_params *p, uint64_t count,
                      const GeomView &gt, uint32_t n_src, int jbits, bool backward,
                      const uint32_t *rx_ids, emrt_paths *out, cudaStream_t st,
                      emrt_paths *merge_cache = nullptr, cudaEvent_t merge_after = nullptr) {
  uint32_t nf = s->Fs + 6 * s->V;
  KeyLayout kl = key_layout(s->n_tx, s->n_rx, nf + 1, (int)p->max_depth);
  if (kl.total > 128) return EMRT_ERR_INVALID_ARG;
  Counters *c = s->ctr;
  // primary direction table of this ray set (built once, kept in an LRU of 4)
  emrt_scene_s::DirTable *tab = nullptr;
  for (auto &t : s->dt)
    if (t.dirs && t.n == p->n_rays && t.off == p->ray_offset && t.stride == p->ray_stride &&
        t.count == count)
      tab = &t;
  if (!tab) {
    tab = &s->dt[0];
    for (auto &t : s->dt)
      if (t.last_use < tab->last_use) tab = &t;
    CK(grow(&tab->dirs, tab->cap, count));
    tab->stab_slots = 0;  // a new ray set: its static-hit cache starts empty
    CK(grow(&s->dt_scratch, s->dt_scratch_cap, 4 * count));
    KeyW<1> *k0 = reinterpret_cast<KeyW<1> *>(s->dt_scratch), *k1 = k0 + count;
    uint32_t *v0 = s->dt_scratch + 2 * count, *v1 = v0 + count;
    build_dir_table(p->n_rays, p->ray_offset, p->ray_stride, (uint32_t)count, tab->dirs, k0, k1,
                    v0, v1, &c->tmp, s->hist, st);
    tab->n = p->n_rays;
    tab->off = p->ray_offset;
    tab->stride = p->ray_stride;
    tab->count = (uint32_t)count;
  }
  tab->last_use = ++s->dt_clock;
  uint64_t nrays = count * n_src;
  // the static-hit cache form runs in the chain walker alone: no per-bounce
  // ray buffers or sorts
  const bool cache = (p->flags & EMRT_TRACE_STATIC_CACHE) && !backward;
  // depth-first chains unless the breadth-first form is asked for
  const bool walk = !cache && !(p->flags & EMRT_TRACE_BREADTH_FIRST);
  if (!cache && !walk && p->max_depth > 0 && nrays > s->ray_cap) {
    cudaFree(s->rays[0]);
    cudaFree(s->rays[1]);
    s->rays[0] = s->rays[1] = nullptr;
    s->ray_cap = 0;
    CK(cudaMalloc(&s->rays[0], sizeof(Ray) * nrays));
    CK(cudaMalloc(&s->rays[1], sizeof(Ray) * nrays));
    s->ray_cap = nrays;
  }
  bool sort_rays = (p->flags & EMRT_TRACE_SORT_RAYS) && p->max_depth > 0 && !cache && !walk;
  if (sort_rays && nrays > s->rsort_cap) {
    for (int k = 0; k < 2; k++) {
      cudaFree(s->rkeys[k]);
      cudaFree(s->rvals[k]);
      s->rkeys[k] = nullptr;
      s->rvals[k] = nullptr;
    }
    s->rsort_cap = 0;
    for (int k = 0; k < 2; k++) {
      CK(cudaMalloc(&s->rkeys[k], sizeof(KeyW<1>) * nrays));
      CK(cudaMalloc(&s->rvals[k], sizeof(uint32_t) * nrays));
    }
    s->rsort_cap = nrays;
  }
  if (cache) {
    const uint32_t depth = p->max_depth + 1;
    if (tab->stab_slots != nrays || tab->stab_depth < depth || !tab->stab) {
      const uint64_t need = nrays * depth;
      if (need > tab->stab_cap) {
        cudaFree(tab->stab);
        tab->stab = nullptr;
        tab->stab_cap = 0;
        CK(cudaMalloc(&tab->stab, sizeof(uint4) * need));
        tab->stab_cap = need;
      }
      if (!tab->tx_ref) CK(cudaMalloc(&tab->tx_ref, sizeof(float4) * s->max_tx));
      if (!tab->tx_epoch) CK(cudaMalloc(&tab->tx_epoch, sizeof(uint32_t) * s->max_tx));
      // epochs restart at 0 and every entry at epoch 0: nothing is current
      // until the epoch kernel has seen the transmitter positions
      cudaMemsetAsync(tab->stab, 0, sizeof(uint4) * need, st);
      cudaMemsetAsync(tab->tx_ref, 0xff, sizeof(float4) * s->max_tx, st);
      cudaMemsetAsync(tab->tx_epoch, 0, sizeof(uint32_t) * s->max_tx, st);
      tab->stab_slots = nrays;
      tab->stab_depth = depth;
    }
    if (!s->chain_q) {
      CK(cudaMalloc(&s->chain_q, sizeof(Ray) * chain_queue_entries()));
    }
  }
  uint64_t want = std::max<uint64_t>(s->want_cand,
                                     std::max<uint64_t>(1u << 16, 4ull * s->n_tx * s->n_rx * (p->max_depth + 1)));
  // a rediscovery also concatenates the cache with the new paths in the
  // candidate scratch
  want = merge_cache ? want + out->capacity : std::max<uint64_t>(want, out->capacity);
  CK(ensure_cand(s, want));
  // counters: keep the error word, clear the rest
  cudaMemsetAsync(reinterpret_cast<char *>(c) + sizeof(uint32_t), 0,
                  sizeof(Counters) - sizeof(uint32_t), st);
  GeomView g = geom(s);
  float kappa = (float)(1.25 * sqrt(8.0 * 3.14159265358979323846 /
                                    (3.0 * sqrt(3.0) * (double)p->n_rays)));
  int grid = bounce_grid();
  cudaEventRecord(s->ev[0], st);
  uint32_t nev = 0;  // traversal launches timed
  if (cache) {
    // static-hit cache: epochs of the transmitter positions, then the chain
    // walker, which also carries the chains it defers to their ends
    launch_tx_epoch(s->tx_pos, tab->tx_ref, tab->tx_epoch, s->n_tx, st);
    BounceLaunch L{};
    L.g = gt;
    L.n_primary = (uint32_t)nrays;
    L.dirs = tab->dirs;
    L.count = (uint32_t)count;
    L.cand = s->cand;
    L.cand_cap = s->cand_cap;
    L.n_cand = &c->n_cand;
    L.work = &c->chain_work;
    L.ctr = c;
    L.kappa = kappa;
    L.K = (int)p->max_depth;
    L.jbits = jbits;
    L.stab = tab->stab;
    L.tx_epoch = tab->tx_epoch;
    L.n_slots = (uint32_t)nrays;
    ChainBufs D{s->chain_q};
    cudaEventRecord(s->evb[0], st);
    launch_chain(L, D, chain_grid(), st);
    cudaEventRecord(s->evb[1], st);
    nev = 1;
  }
  if (walk) {
    BounceLaunch L{};
    L.g = gt;
    L.n_primary = (uint32_t)nrays;
    L.dirs = tab->dirs;
    L.count = (uint32_t)count;
    L.cand = s->cand;
    L.cand_cap = s->cand_cap;
    L.n_cand = &c->n_cand;
    L.work = &c->chain_work;
    L.ctr = c;
    L.kappa = kappa;
    L.K = (int)p->max_depth;
    L.jbits = jbits;
    cudaEventRecord(s->evb[0], st);
    launch_walk(L, st, (p->flags & EMRT_TRACE_WIDE_BVH) != 0);
    cudaEventRecord(s->evb[1], st);
    nev = 1;
  }
  int key_buf = 0;  // sort buffer that receives the next bounce's keys
  for (uint32_t b = 0; !cache && !walk && b <= p->max_depth; b++) {
    BounceLaunch L{};
    L.g = gt;
    L.rin = b ? s->rays[(b - 1) & 1] : nullptr;
    L.order = nullptr;
    // reorder reflected rays for coherent traversal (keys written by the
    // previous bounce into key_buf)
    if (b > 0 && sort_rays) {
      const int o = key_buf, q = 1 - key_buf;
      bool alt = radix_sort<1>(&c->n_ray[b], s->rkeys[o], s->rvals[o], s->rkeys[q], s->rvals[q],
                               24, s->hist, st, nrays);
      const int res = alt ? q : o;
      L.order = s->rvals[res];
      key_buf = 1 - res;  // the next keys go to the buffer not read as order
    }
    L.n_in = &c->n_ray[b];
    L.n_primary = (uint32_t)nrays;
    L.dirs = tab->dirs;
    L.count = (uint32_t)count;
    L.rout = s->rays[b & 1];
    L.n_out = &c->n_ray[b + 1];
    L.cand = s->cand;
    L.cand_cap = s->cand_cap;
    L.n_cand = &c->n_cand;
    L.work = &c->work[b];
    L.ctr = c;
    L.kappa = kappa;
    L.b = (int)b;
    L.K = (int)p->max_depth;
    L.jbits = jbits;
    if (sort_rays && b < p->max_depth) {
      L.okeys = s->rkeys[key_buf];
      L.ovals = s->rvals[key_buf];
      L.bbox = s->bbox;
    }
    cudaEventRecord(s->evb[2 * nev], st);
    launch_bounce(L, grid, st, (p->flags & EMRT_TRACE_WIDE_BVH) != 0);
    cudaEventRecord(s->evb[2 * nev + 1], st);
    nev++;
  }
  s->ev_bounces = nev;
  cudaEventRecord(s->ev[1], st);
  emrt::note_launch(), k_check_cand<<<1, 1, 0, st>>>(c, s->cand_cap);
  if (backward) launch_reverse_candidates(s->cand, &c->n_cand, s->cand_cap, rx_ids, st);
  dedup(s, s->cand, &c->n_cand, s->cand_cap, kl, st);
  cudaEventRecord(s->ev[2], st);
  if (merge_cache) {
    if (merge_after) {  // the cache's revalidation on the side stream
      CK(cudaStreamWaitEvent(st, merge_after, 0));
      emrt::note_launch(), k_fold_counters<<<1, 1, 0, st>>>(s->rv_ctr, c);
    }
    rediscover_tail(s, g, merge_cache, st);
    cudaEventRecord(s->ev[3], st);
    s->ev_recorded = true;
    CK(cudaGetLastError());
    return EMRT_OK;
  }
  launch_accept(g, s->uniq, &c->n_unique, c, s->apts, s->cand_cap, st);
  launch_keep_flags(s->uniq, &c->n_unique, (p->flags & EMRT_TRACE_KEEP_REJECTED) ? 1 : 0, s->head,
                    st);
  exclusive_scan(&c->n_unique, s->head, s->pos, &c->n_accepted, s->partial, st);
  launch_scatter(s->uniq, &c->n_unique, s->head, s->pos, out->rec, out->capacity, &c->n_accepted,
                 c, st);
  emrt::note_launch(), k_publish_count<<<1, 1, 0, st>>>(c, out->count);
  cudaEventRecord(s->ev[3], st);
  s->ev_recorded = true;
  CK(cudaGetLastError());
  return EMRT_OK;
}

// Rays per source of a trace call (0 when the parameters are invalid).
uint64_t ray_count(const emrt_trace_params *p) {
  if (p->max_depth > EMRT_MAX_DEPTH || p->n_rays == 0 || p->ray_stride == 0 ||
      p->ray_offset >= p->n_rays)
    return 0;
  uint64_t count = p->ray_count ? p->ray_count
                                : (p->n_rays - p->ray_offset + p->ray_stride - 1) / p->ray_stride;
  if (count == 0 || p->ray_offset + (count - 1) * p->ray_stride >= p->n_rays) return 0;
  return count;
}

}  // namespace

extern "C" {

emrt_status emrt_trace(emrt_scene s, const emrt_trace_params *p, emrt_paths *out,
                       emrt_stream stream) {
  if (!s || !p || check_paths(out) != EMRT_OK) return EMRT_ERR_INVALID_ARG;
  if (!s->updated) return EMRT_ERR_STATE;
  uint64_t count = ray_count(p);
  if (count == 0 || count > (1u << 24) || count * s->n_tx >= (1ull << 32))
    return EMRT_ERR_INVALID_ARG;
  return run_trace(s, p, count, geom(s), s->n_tx, 24, false, nullptr, out,
                   (cudaStream_t)stream);
}

emrt_status emrt_rediscover(emrt_scene s, const emrt_trace_params *p, emrt_paths *cache,
                            emrt_stream stream) {
  if (!s || !p || check_paths(cache) != EMRT_OK) return EMRT_ERR_INVALID_ARG;
  if (p->flags & EMRT_TRACE_KEEP_REJECTED) return EMRT_ERR_INVALID_ARG;
  if (!s->updated) return EMRT_ERR_STATE;
  uint64_t count = ray_count(p);
  if (count == 0 || count > (1u << 24) || count * s->n_tx >= (1ull << 32))
    return EMRT_ERR_INVALID_ARG;
  const uint32_t nf = s->Fs + 6 * s->V;
  if (key_layout(s->n_tx, s->n_rx, nf + 1, EMRT_MAX_DEPTH).total > 128) return EMRT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t after = nullptr;
  if (p->flags & EMRT_TRACE_REVALIDATE_FIRST) {
    // revalidate the cache on a side stream while the discovery runs; the
    // merge waits for it
    CK(ensure_rv(s, cache->capacity));
    CK(cudaEventRecord(s->ev_fork, st));
    CK(cudaStreamWaitEvent(s->side[0], s->ev_fork, 0));
    cudaMemsetAsync(s->rv_ctr, 0, sizeof(Counters), s->side[0]);
    revalidate_with(s, cache, 0u, s->side[0], s->rv_rec, s->rv_head, s->rv_pos, s->rv_partial,
                    s->rv_apts, (uint32_t)s->rv_cap, s->rv_ctr);
    CK(cudaEventRecord(s->ev_side[0], s->side[0]));
    after = s->ev_side[0];
  }
  const emrt_status r =
      run_trace(s, p, count, geom(s), s->n_tx, 24, false, nullptr, cache, st, cache, after);
  // whatever run_trace returned (an early return skips its merge, which
  // waits for the revalidation), the caller's stream is ordered after the
  // side stream's writes to the cache
  if (after) cudaStreamWaitEvent(st, after, 0);
  return r;
}

emrt_status emrt_trace_backward(emrt_scene s, const emrt_trace_params *p, const uint32_t *rx_ids,
                                uint32_t n_ids, emrt_paths *out, emrt_stream stream) {
  if (!s || !p || check_paths(out) != EMRT_OK) return EMRT_ERR_INVALID_ARG;
  if (!s->updated) return EMRT_ERR_STATE;
  const uint32_t n_src = rx_ids ? n_ids : s->n_rx;
  if (n_src == 0 || n_src > s->n_rx) return EMRT_ERR_INVALID_ARG;
  uint64_t count = ray_count(p);
  const int jbits = 32 - id_bits(n_src);
  if (count == 0 || count > (1ull << jbits) || count * n_src >= (1ull << 32))
    return EMRT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  GeomView gb = geom(s);
  if (rx_ids) {
    CK(grow(&s->src_pos, s->src_cap, n_src));
    launch_gather_points(s->rx_pos, rx_ids, n_src, s->src_pos, st);
    gb.tx_pos = s->src_pos;
  } else {
    gb.tx_pos = s->rx_pos;
  }
  CK(bvh_build_points(s->txb, s->tx_pos, s->n_tx, s->bbox, s->hist, st));
  gb.rxb = s->txb.view();
  gb.mix = BVHView{};  // backward: the transmitters take the receivers' place
  gb.n_tx = n_src;
  gb.n_rx = s->n_tx;
  return run_trace(s, p, count, gb, n_src, jbits, true, rx_ids, out, st);
}

emrt_status emrt_revalidate(emrt_scene s, emrt_paths *cache, uint32_t flags, emrt_stream stream) {
  if (!s || check_paths(cache) != EMRT_OK) return EMRT_ERR_INVALID_ARG;
  if (!s->updated) return EMRT_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  CK(ensure_cand(s, std::max<uint64_t>(s->want_cand, cache->capacity)));
  revalidate_with(s, cache, flags, st, s->uniq, s->head, s->pos, s->partial, s->apts, s->cand_cap,
                  s->ctr);
  CK(cudaGetLastError());
  return EMRT_OK;
}

emrt_status emrt_revalidate_cache(emrt_scene s, emrt_paths *cache, uint32_t *n_evicted,
                                  emrt_stream stream) {
  emrt_status e = emrt_revalidate(s, cache, 0u, stream);
  if (e != EMRT_OK || !n_evicted) return e;
  launch_evicted(s->ctr, n_evicted, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return EMRT_OK;
}

emrt_status emrt_cache_merge(emrt_scene s, emrt_paths *cache, const emrt_paths *fresh,
                             emrt_stream stream) {
  if (!s || check_paths(cache) != EMRT_OK || check_paths(fresh) != EMRT_OK)
    return EMRT_ERR_INVALID_ARG;
  if (!s->updated) return EMRT_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  CK(ensure_cand(s, std::max<uint64_t>(s->want_cand,
                                       (uint64_t)cache->capacity + fresh->capacity)));
  Counters *c = s->ctr;
  uint32_t nf = s->Fs + 6 * s->V;
  KeyLayout kl = key_layout(s->n_tx, s->n_rx, nf + 1, EMRT_MAX_DEPTH);
  if (kl.total > 128) return EMRT_ERR_INVALID_ARG;
  launch_concat(cache->rec, cache->count, cache->capacity, fresh->rec, fresh->count,
                fresh->capacity, s->cand, s->cand_cap, &c->tmp, c, st);
  // both inputs are in canonical order: merge their keys along the merge
  // path instead of sorting the concatenation, then merge equal runs
  launch_path_keys(s->cand, &c->tmp, s->cand_cap, kl, s->keys[0], s->vals[0], &c->n_eff, st);
  launch_merge_path(s->keys[0], s->vals[0], cache->count, cache->capacity, &c->n_eff, s->keys[1],
                    s->vals[1], c, st);
  launch_heads(s->keys[1], &c->n_eff, s->head, st);
  exclusive_scan(&c->n_eff, s->head, s->pos, &c->n_unique, s->partial, st);
  launch_unique(s->cand, s->keys[1], s->vals[1], s->head, s->pos, &c->n_eff, s->uniq, st);
  launch_keep_flags(s->uniq, &c->n_unique, 1, s->head, st);
  exclusive_scan(&c->n_unique, s->head, s->pos, &c->n_accepted, s->partial, st);
  launch_scatter(s->uniq, &c->n_unique, s->head, s->pos, cache->rec, cache->capacity,
                 &c->n_accepted, c, st);
  emrt::note_launch(), k_publish_count<<<1, 1, 0, st>>>(c, cache->count);
  CK(cudaGetLastError());
  return EMRT_OK;
}

static emrt_status check_mat(const emrt_materials *m) {
  if (!m || m->n_mat == 0 || !m->eps_r || !m->sigma || (m->const_gamma && !m->gamma))
    return EMRT_ERR_INVALID_ARG;
  return EMRT_OK;
}

static MatView matview(const emrt_materials *m) {
  MatView v;
  v.eps_r = m->eps_r;
  v.sigma = m->sigma;
  v.gamma = m->gamma;
  v.n_mat = m->n_mat;
  v.const_gamma = m->const_gamma;
  return v;
}

emrt_status emrt_channel(emrt_scene s, const emrt_paths *paths, const emrt_materials *m,
                         double freq_hz, double tx_power_w, emrt_channel_out *out,
                         emrt_stream stream) {
  if (!out) return EMRT_ERR_INVALID_ARG;
  return emrt_channel_multi(s, paths, m, &freq_hz, 1, tx_power_w, out, stream);
}

emrt_status emrt_channel_multi(emrt_scene s, const emrt_paths *paths, const emrt_materials *m,
                               const double *freq_hz, uint32_t n_freq, double tx_power_w,
                               emrt_channel_out *outs, emrt_stream stream) {
  if (!s || check_paths(paths) != EMRT_OK || check_mat(m) != EMRT_OK || !freq_hz || !outs ||
      n_freq == 0 || n_freq > kMaxFreq)
    return EMRT_ERR_INVALID_ARG;
  FreqSet fs{};
  fs.n = n_freq;
  for (uint32_t q = 0; q < n_freq; q++) {
    if (!outs[q].path_out || !outs[q].pair_out || !(freq_hz[q] > 0)) return EMRT_ERR_INVALID_ARG;
    fs.f[q] = freq_hz[q];
    fs.path_out[q] = outs[q].path_out;
    fs.pair_out[q] = outs[q].pair_out;
    fs.rx_out[q] = outs[q].rx_out;
  }
  if (!s->updated) return EMRT_ERR_STATE;
  launch_channel(geom(s), matview(m), paths->rec, paths->count, paths->capacity, fs, s->n_tx,
                 s->n_rx, tx_power_w, s->ctr, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return EMRT_OK;
}

emrt_status emrt_channel_backward(emrt_scene s, const emrt_paths *paths, const emrt_materials *m,
                                  double freq_hz, const double *dloss_dh, double *grad_eps,
                                  double *grad_sigma, double *grad_tx, emrt_stream stream) {
  if (!s || check_paths(paths) != EMRT_OK || check_mat(m) != EMRT_OK || !dloss_dh || !grad_eps ||
      !grad_sigma || !grad_tx || !(freq_hz > 0))
    return EMRT_ERR_INVALID_ARG;
  if (!s->updated) return EMRT_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  uint64_t need = (uint64_t)paths->capacity * (3 + 2 * EMRT_MAX_DEPTH);
  CK(grow(&s->contrib, s->contrib_cap, std::max<uint64_t>(need, s->contrib_cap)));
  GeomView g = geom(s);
  launch_field_adjoint(g, matview(m), paths->rec, paths->count, paths->capacity, freq_hz, dloss_dh,
                       s->n_rx, s->contrib, grad_eps, grad_sigma, grad_tx, s->ctr, st);
  CK(cudaGetLastError());
  return EMRT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free adjoint: the per-path tangent scratch is this file-scope
// device array (EMRT_NOALLOC_MAX_PATHS x 11 doubles).  Host code must not use
// the symbol `g_noalloc_contrib` as an address: it is a host-side stand-in.
// Its device address is looked up once per device, with that device current,
// by noalloc_scratch() and cached here.
static __device__ __align__(256) double
    g_noalloc_contrib[(size_t)EMRT_NOALLOC_MAX_PATHS * (3 + 2 * EMRT_MAX_DEPTH)];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kMaxDevices] = {};

cudaError_t noalloc_scratch(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_contrib);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}
}  // namespace

extern "C" {

emrt_status emrt_channel_backward_noalloc(emrt_scene s, const emrt_paths *paths,
                                          const emrt_materials *m, double freq_hz,
                                          const double *dloss_dh, double *grad_eps,
                                          double *grad_sigma, double *grad_tx,
                                          emrt_stream stream) {
  if (!s || check_paths(paths) != EMRT_OK || check_mat(m) != EMRT_OK || !dloss_dh || !grad_eps ||
      !grad_sigma || !grad_tx || !(freq_hz > 0))
    return EMRT_ERR_INVALID_ARG;
  if (paths->capacity > EMRT_NOALLOC_MAX_PATHS) return EMRT_ERR_INVALID_ARG;
  if (!s->updated) return EMRT_ERR_STATE;
  double *scratch = nullptr;
  CK(noalloc_scratch(&scratch));
  cudaStream_t st = (cudaStream_t)stream;
  GeomView g = geom(s);
  launch_field_adjoint(g, matview(m), paths->rec, paths->count, paths->capacity, freq_hz, dloss_dh,
                       s->n_rx, scratch, grad_eps, grad_sigma, grad_tx, s->ctr, st);
  CK(cudaGetLastError());
  return EMRT_OK;
}

emrt_status emrt_channel_correlation(const double *h, uint32_t n_frames, uint32_t n_pairs,
                                     uint32_t max_lag, double *R, emrt_stream stream) {
  if (!h || !R || n_frames == 0 || n_pairs == 0) return EMRT_ERR_INVALID_ARG;
  launch_correlation(h, n_frames, n_pairs, max_lag, R, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return EMRT_OK;
}

emrt_status emrt_coherence_time(emrt_scene s, double freq_hz, double r_threshold, double *tc,
                                emrt_stream stream) {
  if (!s || !tc || !(freq_hz > 0) || !(r_threshold > 0) || !(r_threshold <= 1))
    return EMRT_ERR_INVALID_ARG;
  if (!s->updated) return EMRT_ERR_STATE;
  launch_coherence(emrt::geom(s), freq_hz, r_threshold, tc, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return EMRT_OK;
}

emrt_status emrt_refresh_schedule(emrt_scene s, float *state, uint8_t *los_ref, double freq_hz,
                                  double r_threshold, double dt_s, float d_seg,
                                  uint32_t max_interval, uint32_t *ids, uint32_t *n_due,
                                  emrt_stream stream) {
  if (!s || !state || !los_ref || !ids || !n_due || !(freq_hz > 0) || !(r_threshold > 0) ||
      !(r_threshold <= 1) || !(dt_s >= 0) || !(d_seg >= 0) || max_interval == 0)
    return EMRT_ERR_INVALID_ARG;
  if (!s->updated) return EMRT_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t pairs = (uint64_t)s->n_tx * s->n_rx;
  CK(ensure_cand(s, std::max<uint64_t>(s->want_cand, pairs)));
  Counters *c = s->ctr;
  GeomView g = geom(s);
  // line of sight of every pair: its direct path through the acceptance
  // kernel (occlusion by static faces and vehicle boxes, same margins)
  launch_los_records(s->n_tx, s->n_rx, s->uniq, st);
  launch_set_u32(&c->tmp, (uint32_t)pairs, st);
  launch_accept(g, s->uniq, &c->tmp, c, s->apts, s->cand_cap, st);
  launch_schedule(g, s->uniq, reinterpret_cast<float4 *>(state), los_ref, freq_hz, r_threshold,
                  dt_s, d_seg, max_interval, s->head, st);
  launch_set_u32(&c->tmp, s->n_rx, st);
  exclusive_scan(&c->tmp, s->head, s->pos, n_due, s->partial, st);
  launch_compact_ids(s->head, s->pos, s->n_rx, ids, st);
  CK(cudaGetLastError());
  return EMRT_OK;
}

emrt_status emrt_sync(emrt_scene s, emrt_stream stream, emrt_stats *out) {
  if (!s) return EMRT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaStreamSynchronize(st));
  Counters h;
  CK(cudaMemcpy(&h, s->ctr, sizeof(Counters), cudaMemcpyDeviceToHost));
  CK(cudaMemset(s->ctr, 0, sizeof(uint32_t)));
  if (h.n_cand > s->cand_cap) s->want_cand = (uint32_t)std::min<uint64_t>(
      (uint64_t)h.n_cand + h.n_cand / 4 + 1024, 0x7fffffffull);
  if (out) {
    memset(out, 0, sizeof(*out));
    for (int b = 0; b <= EMRT_MAX_DEPTH; b++) out->segments[b] = h.segments[b];
    out->candidates = h.n_cand;
    out->unique_candidates = h.n_unique;
    out->accepted = h.n_accepted;
    out->occlusion_rays = h.occl_rays;
    out->node_visits = h.node_visits;
    out->tri_tests = h.tri_tests;
    out->error_bits = h.err;
    out->dyn_node_visits = h.dyn_node_visits;
    out->box_tests = h.box_tests;
    out->rx_node_visits = h.rx_node_visits;
    out->rx_tests = h.rx_tests;
    out->static_reused = h.static_reused;
    out->deferred = h.deferred;
    if (s->ev_recorded) {
      cudaEventElapsedTime(&out->traverse_ms, s->ev[0], s->ev[1]);
      cudaEventElapsedTime(&out->dedup_ms, s->ev[1], s->ev[2]);
      cudaEventElapsedTime(&out->accept_ms, s->ev[2], s->ev[3]);
      cudaEventElapsedTime(&out->trace_ms, s->ev[0], s->ev[3]);
      out->bounce_ms = 0.f;
      for (uint32_t b = 0; b < s->ev_bounces; b++) {
        float t = 0.f;
        cudaEventElapsedTime(&t, s->evb[2 * b], s->evb[2 * b + 1]);
        out->bounce_ms += t;
      }
      // a trace recorded into a caller's CUDA graph leaves these events
      // without a time: the query's error is dropped, not reported later
      (void)cudaGetLastError();
    }
    out->required_candidates = h.n_cand;
    out->required_paths = h.n_accepted;
  }
  emrt_status r = s->sticky;
  s->sticky = EMRT_OK;
  if (r != EMRT_OK) return r;
  if (h.err & ERR_WAIT) return EMRT_ERR_TIMEOUT;
  if (h.err & (ERR_STACK | ERR_NONFINITE)) return EMRT_ERR_DEVICE;
  if (h.err & ERR_UNSORTED) return EMRT_ERR_INVALID_ARG;
  if (h.err & (ERR_CAND_OVERFLOW | ERR_PATH_OVERFLOW | ERR_RAY_OVERFLOW)) return EMRT_ERR_CAPACITY;
  return EMRT_OK;
}

}  // extern "C"
