// Internal definition of the scene object shared by the C-ABI translation
// units (api.cu, batch.cu).
#pragma once
#include "bvh.cuh"
#include "trace.cuh"

using namespace emrt;  // internal header: included by the C-ABI units only

struct emrt_scene_s {
  int device = 0;
  uint32_t Fs = 0, T = 0, V = 0, NV = 0, max_rx = 0, max_tx = 0, veh_mat = 0;
  uint32_t rebuild_every = 1, n_updates = 0;
  double4_32a *face_plane = nullptr;
  uint4 *face_info = nullptr;
  float4 *face_vert = nullptr;
  float4 *bbox = nullptr;  // [4]: lo, hi, scratch
  BVHBuf stat, dyn, rxb;
  BVHBuf txb;                     // transmitter points (backward tracing)
  BVHBuf mix;                     // vehicles + receivers (merged per-frame tree)
  float4 *mix_lo = nullptr, *mix_hi = nullptr;  // its primitive corners
  float4 *src_pos = nullptr;      // receiver points shot from (backward tracing)
  uint64_t src_cap = 0;
  float4 *veh_half = nullptr, *veh_lo = nullptr, *veh_hi = nullptr, *veh_vel = nullptr;
  float4 *rx_pos = nullptr, *rx_vel = nullptr, *tx_pos = nullptr, *tx_vel = nullptr;
  uint32_t n_rx = 0, n_tx = 0;
  bool updated = false;
  Counters *ctr = nullptr;
  uint32_t *hist = nullptr, *partial = nullptr;
  // primary direction tables, one per recently used ray set (LRU)
  struct DirTable {
    uint64_t n = 0, off = 0, stride = 0, cap = 0, last_use = 0;
    uint32_t count = 0;
    float4 *dirs = nullptr;
    // static-hit cache of this ray set: (depth) x (slots) entries, transmitter
    // positions they were computed for and their epochs
    uint4 *stab = nullptr;
    uint64_t stab_cap = 0, stab_slots = 0;
    uint32_t stab_depth = 0;
    float4 *tx_ref = nullptr;
    uint32_t *tx_epoch = nullptr;
  } dt[4];
  uint64_t dt_clock = 0;
  uint32_t *dt_scratch = nullptr;  // key/value scratch for building a table
  uint64_t dt_scratch_cap = 0;
  // ray ping-pong buffers and the coherence-sort scratch
  Ray *rays[2] = {nullptr, nullptr};
  uint64_t ray_cap = 0;
  // per-warp deferred-chain queues of the static-hit cache walker
  Ray *chain_q = nullptr;
  KeyW<1> *rkeys[2] = {nullptr, nullptr};
  uint32_t *rvals[2] = {nullptr, nullptr};
  uint64_t rsort_cap = 0;
  // candidate and path scratch
  uint32_t cand_cap = 0, want_cand = 0;
  uint32_t *cand = nullptr, *uniq = nullptr, *head = nullptr, *pos = nullptr;
  float4 *apts = nullptr;  // acceptance scratch: reflection points, point-major
  KeyW<4> *keys[2] = {nullptr, nullptr};
  uint32_t *vals[2] = {nullptr, nullptr};
  // adjoint scratch
  double *contrib = nullptr;
  uint64_t contrib_cap = 0;
  emrt_status sticky = EMRT_OK;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // revalidation scratch of a rediscovery that revalidates its cache on a
  // side stream while the discovery runs: records, flags, positions, scan
  // partials, reflection points (capacity rv_cap) and its own counters
  uint32_t *rv_rec = nullptr, *rv_head = nullptr, *rv_pos = nullptr, *rv_partial = nullptr;
  float4 *rv_apts = nullptr;
  Counters *rv_ctr = nullptr;
  uint64_t rv_cap = 0;
  // side streams of the per-frame tree builds (vehicles, receivers), their
  // fork/join events and histogram scratch
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_side[2] = {nullptr, nullptr};
  uint32_t *hist_side[2] = {nullptr, nullptr};
  cudaEvent_t evb[2 * (EMRT_MAX_DEPTH + 2)] = {};  // around each traversal launch
  uint32_t ev_bounces = 0;
  bool ev_recorded = false;
};


// batch.cu: discards the emrt_trace_batched batches that use scene s
void batch_forget_scene(emrt_scene s);

namespace emrt {
inline GeomView geom(const emrt_scene_s *s) {
  GeomView g;
  g.stat = s->stat.view();
  g.dyn = s->dyn.view();
  g.rxb = s->rxb.view();
  g.mix = s->mix.view();
  g.face_plane = s->face_plane;
  g.face_info = s->face_info;
  g.face_vert = s->face_vert;
  g.veh_lo = s->veh_lo;
  g.veh_hi = s->veh_hi;
  g.veh_vel = s->veh_vel;
  g.rx_pos = s->rx_pos;
  g.rx_vel = s->rx_vel;
  g.tx_pos = s->tx_pos;
  g.tx_vel = s->tx_vel;
  g.n_static_faces = s->Fs;
  g.n_veh = s->V;
  g.n_rx = s->n_rx;
  g.n_tx = s->n_tx;
  g.veh_mat = s->veh_mat;
  return g;
}

}  // namespace emrt
