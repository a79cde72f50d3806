// Host launchers of the discovery and acceptance kernels.
#pragma once
#include "common.cuh"
#include "prims.cuh"

namespace emrt {

struct KeyLayout {  // bit widths of the canonical 128-bit path key
  int bs, bt, br, bf, K, total;  // bs: scene bits (batches), 0 otherwise
};
KeyLayout key_layout(uint32_t n_tx, uint32_t n_rx, uint32_t n_faces, int K,
                     uint32_t n_scenes = 1);

// Primary direction table for rays offset + stride*j, j < count: float4
// (unit direction, j bits), ordered by an octahedral direction code so that
// neighbouring threads shoot neighbouring directions.
void build_dir_table(uint64_t n_rays, uint64_t offset, uint64_t stride, uint32_t count,
                     float4 *table, KeyW<1> *k0, KeyW<1> *k1, uint32_t *v0, uint32_t *v1,
                     uint32_t *d_n, uint32_t *hist, cudaStream_t s);

struct BounceLaunch {
  GeomView g;
  const Ray *rin;        // bounce >= 1
  const uint32_t *order; // optional permutation of rin (coherence sort)
  const uint32_t *n_in;  // device count of rin (bounce >= 1)
  uint32_t n_primary;    // n_tx * count (bounce 0)
  const float4 *dirs;
  uint32_t count;
  Ray *rout;
  uint32_t *n_out;
  uint32_t *cand;
  uint32_t cand_cap;
  uint32_t *n_cand;
  uint32_t *work;
  Counters *ctr;
  float kappa;
  int b, K;
  int jbits;             // single-scene ray ids: source << jbits | ray index j
  // static-hit cache (chain walker): entry (bounce b, item i) at
  // stab[b * n_slots + i], item i = tx * count + position in the direction
  // table; uint4 (t bits, face, epoch of the tx position, 0).  The walker's
  // ray ids carry the direction-table position instead of j.
  uint4 *stab;
  const uint32_t *tx_epoch;
  uint32_t n_slots;
  // optional (single scene): coherence key and index of every reflected ray
  // written, at the ray's slot, for the next bounce's sort (box: scene bbox)
  KeyW<1> *okeys;
  uint32_t *ovals;
  const float4 *bbox;
};
// Per-warp queues of the static-hit cache walker: warp w of the launch owns
// q[w * kChainQueue, (w + 1) * kChainQueue); chain_queue_entries() entries in
// all for chain_grid() blocks.
constexpr uint32_t kChainQueue = 64;
struct ChainBufs {
  Ray *q;
};
uint64_t chain_queue_entries();
void launch_chain(const BounceLaunch &L, const ChainBufs &D, int grid, cudaStream_t s);
int chain_grid();
// Depth-first discovery of L.n_primary primary rays without the cache
// (persistent grid; cursor L.work); wide: static closest hits through the
// compressed 8-wide tree.
void launch_walk(const BounceLaunch &L, cudaStream_t s, bool wide = false);
// epoch[t] += 1 and ref[t] = pos[t] for every transmitter whose position
// differs (bitwise) from ref[t]
void launch_tx_epoch(const float4 *pos, float4 *ref, uint32_t *epoch, uint32_t n_tx,
                     cudaStream_t s);
// wide: static closest hits through the compressed 8-wide tree
void launch_bounce(const BounceLaunch &L, int grid, cudaStream_t s, bool wide = false);
int bounce_grid();  // persistent grid size (SMs x resident blocks)

// One scene of a batch (device table entry).  Batched rays pack
// scene (6 bits) | tx (4 bits) | ray index (22 bits); batched candidate and
// path records carry scene << 8 | tx in word 0 until they are written to the
// scene's own output.
struct BatchScene {
  GeomView g;
  const float4 *dirs;     // primary direction table of this scene
  uint32_t count;         // rays per transmitter
  uint32_t prim_begin;    // first global primary item of this scene
  uint32_t n_primary;     // n_tx * count
  uint32_t K;             // reflections
  float kappa;            // reception radius factor
  uint32_t *out_rec;      // caller's output records
  uint32_t out_cap;
  uint32_t *out_count;
};
constexpr uint32_t kBatchMaxScenes = 64, kBatchMaxTx = 16, kBatchMaxCount = 1u << 22;

// Batched traversal variants: breadth-first (block size x rays fetched per
// warp, one launch per bounce) and depth-first (block size, one launch for
// all bounces); the autotuner picks one.  variant in [0, n_bounce_variants()).
int n_bounce_variants();
const char *bounce_variant_name(int v);
bool bounce_variant_depth_first(int v);
int default_bounce_variant();  // the variant used without autotuning
int default_breadth_first_variant();  // ... with EMRT_BATCH_BREADTH_FIRST
int bounce_variant_grid(int v);
void launch_bounce_batched(int variant, const BounceLaunch &L, const BatchScene *tab,
                           uint32_t n_scenes, cudaStream_t s);
// pts: scratch of (EMRT_MAX_DEPTH + 2) * cap float4 (reflection points);
// records [0, min(*n, cap))
void launch_accept_batched(const BatchScene *tab, uint32_t *rec, const uint32_t *n, Counters *ctr,
                           float4 *pts, uint32_t cap, cudaStream_t s);
// writes kept, sorted batched records to each scene's output (positions
// relative to the scene's first kept record); first[] and cnt[] are
// kBatchMaxScenes words of scratch
void launch_batch_scatter(const BatchScene *tab, uint32_t n_scenes, const uint32_t *rec,
                          const uint32_t *n, const uint32_t *flag, const uint32_t *pos,
                          uint32_t *first, uint32_t *cnt, Counters *ctr, cudaStream_t s);

// Coherence keys of the *n rays (24 bits, three radix passes): origin cell
// (5-bit Morton per axis in the scene box) then direction bin (9 bits of the
// octahedral code).
// batched (24 bits): scene (6) | origin cell (4-bit Morton per axis, 12) |
// direction bin (6)
void launch_ray_keys(const Ray *r, const uint32_t *n, const float4 *bbox, KeyW<1> *keys,
                     uint32_t *vals, cudaStream_t s, bool batched = false);

// Canonical keys of min(*n, cap) records; values = record index.
void launch_path_keys(const uint32_t *rec, const uint32_t *n, uint32_t cap, KeyLayout kl,
                      KeyW<4> *keys, uint32_t *vals, uint32_t *n_eff, cudaStream_t s);
// head[i] = 1 where sorted key i starts a run.
void launch_heads(const KeyW<4> *keys, const uint32_t *n, uint32_t *head, cudaStream_t s);
// uniq[pos[i]] = merged record of the run starting at i (smallest ray index).
void launch_unique(const uint32_t *rec, const KeyW<4> *keys, const uint32_t *vals,
                   const uint32_t *head, const uint32_t *pos, const uint32_t *n, uint32_t *uniq,
                   cudaStream_t s);
// Image-method acceptance and occlusion of min(*n, cap) records in place
// (w2 flags); pts: scratch of (EMRT_MAX_DEPTH + 2) * cap float4.
void launch_accept(const GeomView &g, uint32_t *rec, const uint32_t *n, Counters *ctr,
                   float4 *pts, uint32_t cap, cudaStream_t s);
// flag[i] = 1 if record i is kept (valid, or every record when keep_all).
void launch_keep_flags(const uint32_t *rec, const uint32_t *n, int keep_all, uint32_t *flag,
                       cudaStream_t s);
// out[pos[i]] = in[i] for flagged i with pos < cap; raises ERR_PATH_OVERFLOW
// when *total > cap.
void launch_scatter(const uint32_t *in, const uint32_t *n, const uint32_t *flag,
                    const uint32_t *pos, uint32_t *out, uint32_t cap, const uint32_t *total,
                    Counters *ctr, cudaStream_t s);
// out[0..min(*n,cap)) = in; *n_out = *n
void launch_copy_records(const uint32_t *in, const uint32_t *n, uint32_t *out, uint32_t cap,
                         cudaStream_t s);
// concatenation of two record sets into dst (count written to *n_dst)
void launch_concat(const uint32_t *a, const uint32_t *na, uint32_t cap_a, const uint32_t *b,
                   const uint32_t *nb, uint32_t cap_b, uint32_t *dst, uint32_t dst_cap,
                   uint32_t *n_dst, Counters *ctr, cudaStream_t s);
// Stable merge of the canonical key runs keys[0, na) and keys[na, *n)
// (na = min(*na, cap_a, *n); the first run first among equal keys) into
// (kout, vout); ERR_UNSORTED when a run is out of order.
void launch_merge_path(const KeyW<4> *keys, const uint32_t *vals, const uint32_t *na, uint32_t cap_a,
                       const uint32_t *n, KeyW<4> *kout, uint32_t *vout, Counters *ctr,
                       cudaStream_t s);
// flag[i] = 1 for each of the *n canonical candidate records the canonical
// cache (min(*cache_n, cache_cap) records) does not hold; a candidate it holds
// as a valid path lowers that record's smallest ray index (word 7).
void launch_known(const uint32_t *cand, const uint32_t *n, uint32_t *cache, const uint32_t *cache_n,
                  uint32_t cache_cap, KeyLayout kl, uint32_t *flag, cudaStream_t s);
// out[k] = rec[vals[k]] for k < min(*n, cap); ERR_PATH_OVERFLOW when *n > cap.
void launch_gather_records(const uint32_t *rec, const uint32_t *vals, const uint32_t *n,
                           uint32_t *out, uint32_t cap, Counters *ctr, cudaStream_t s);
// Deduplication sorts run radix passes over the top kDedupPasses bytes of
// the canonical key only and then launch_sort_runs (measured on the city:
// 4 passes 0.11 ms, 5 0.13, 6 0.15, all 11 0.22).
constexpr int kDedupPasses = 4;
// Completes a sort of (keys, vals)[0, *n) that is ordered by the key bits
// from low_bits up: runs equal in those bits are sorted by the whole key.
void launch_sort_runs(KeyW<4> *keys, uint32_t *vals, const uint32_t *n, int low_bits,
                      cudaStream_t s);
void launch_set_u32(uint32_t *p, uint32_t v, cudaStream_t s);

// Backward tracing.  out[i] = pos[ids[i]] for i < n (source points of the
// selected receivers).
void launch_gather_points(const float4 *pos, const uint32_t *ids, uint32_t n, float4 *out,
                          cudaStream_t s);
// Candidates found from the receiver side (word 0 = source index, word 1 =
// transmitter, faces in the order met from the receiver) rewritten in place
// in forward orientation: word 0 = transmitter, word 1 = ids[source] (or the
// source index when ids is null), faces reversed; depth, flags and ray index
// kept.  Records [0, min(*n, cap)).
void launch_reverse_candidates(uint32_t *cand, const uint32_t *n, uint32_t cap,
                               const uint32_t *ids, cudaStream_t s);

}  // namespace emrt
