/*
 * emrt — dynamic urban EM ray tracing on one GB300 GPU (arXiv 2303.10521).
 *
 * C-ABI of libemrt.so.  Plain pointers and sizes only.  Unless stated
 * otherwise every array argument is a DEVICE pointer owned by the caller and
 * every call is asynchronous on the given stream (a cudaStream_t passed as
 * void*; NULL = legacy default stream).  Argument errors are returned
 * synchronously.  Errors raised inside kernels (capacity overflow, traversal
 * stack overflow) are recorded in the scene's device error word and returned
 * by emrt_sync.  The scene owns its BVHs and scratch buffers; it allocates
 * them in emrt_scene_create and grows them inside emrt_trace only when a
 * larger problem than before is requested.
 *
 * Method (paper passages): per frame the engine refits a BVH over static
 * building triangles and moving vehicle boxes (Sec. II-A "dynamic BVH",
 * Sec. III-A "only the subtrees need to be rebuilt", Sec. V-A factors 1-2),
 * shoots and bounces rays from each transmitter with reception spheres at
 * every receiver (Sec. II-A: direct and reflected rays), stores paths as
 * face-ID sequences in a cache revalidated every frame (Sec. II-A path
 * caching, Sec. III-B: paths kept and updated until removed), and gives each
 * accepted path its complex field with Fresnel reflection, spreading and the
 * Doppler shift (Sec. III-C, Eq. 3), reduced per receiver into the
 * statistics of Table III (Sec. V-D).
 *
 * Per-frame calls (emrt_scene_update_dynamic, emrt_trace, emrt_rediscover,
 * emrt_revalidate, emrt_cache_merge, emrt_channel, emrt_channel_multi,
 * emrt_batch_trace) allocate only when a problem larger than any before
 * arrives and do not synchronise the host while their stream is being
 * captured; once a call has run with its sizes, the same call can be
 * recorded into a caller's CUDA graph (stream capture) and replayed,
 * reading its inputs from the same device buffers.
 *
 * Geometry conventions
 *  - float32 metres centred on the scene origin, z up.
 *  - Static faces are convex planar polygons (CCW seen from outside); the
 *    triangles of tri_xyz must cover them exactly (tri_face maps each
 *    triangle to its face).  Static face IDs are 0..F_s-1.
 *  - Vehicle v is the axis-aligned box pos - half .. pos + half; its faces
 *    have IDs F_s + 6v + j, j = 0..5 for -x, +x, -y, +y, -z, +z.
 *
 * Path record (8 x uint32, canonical order = lexicographic over w0..w6):
 *   w0 transmitter index, w1 receiver index,
 *   w2 depth (bits 0-3) | EMRT_PATH_* flags (bits 8-15),
 *   w3..w6 face IDs of the reflections in travel order (0xFFFFFFFF unused),
 *   w7 smallest index j of a discovering ray (ray = offset + stride * j).
 */
#ifndef EMRT_H
#define EMRT_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define EMRT_MAX_DEPTH 4
#define EMRT_PATH_WORDS 8
#define EMRT_NO_FACE 0xFFFFFFFFu

/* path flags (w2 bits 8-15) */
#define EMRT_PATH_VALID 0x100u     /* passed image-method acceptance        */
#define EMRT_PATH_MARGINAL 0x200u  /* a reflection point lies within the
                                      margin of its face boundary           */

/* emrt_trace_params.flags */
#define EMRT_TRACE_KEEP_REJECTED 0x1u  /* output every unique candidate, with
                                          EMRT_PATH_VALID set on accepted ones */
#define EMRT_TRACE_SORT_RAYS 0x2u      /* breadth-first form: reorder rays
                                          between bounces by origin cell and
                                          direction bin                       */
#define EMRT_TRACE_WIDE_BVH 0x4u       /* static closest hits through the
                                          compressed 8-wide BVH (8-bit child
                                          boxes on a per-node grid, 80 B per
                                          node; Sec. II-A BVH) instead of the
                                          binary one, in either traversal
                                          form; same results bit for bit   */
#define EMRT_TRACE_STATIC_CACHE 0x8u   /* keep the static-geometry closest hit of
                                          every ray segment between calls (see
                                          emrt_trace); same results bit for bit */
#define EMRT_TRACE_REVALIDATE_FIRST 0x20u /* emrt_rediscover only: revalidate
                                          the cache first (as emrt_revalidate,
                                          compacting), on a side stream while
                                          the discovery runs              */
#define EMRT_TRACE_BREADTH_FIRST 0x10u /* trace bounce by bounce over all rays
                                          (one launch per bounce, rays kept in
                                          buffers between bounces) instead of
                                          the default depth-first chains (32
                                          neighbouring primary rays per warp,
                                          each carried to its end); same
                                          results bit for bit                 */
/* emrt_revalidate flags */
#define EMRT_REVALIDATE_KEEP 0x1u      /* do not compact: flag only          */

typedef void *emrt_stream; /* cudaStream_t */

typedef enum {
  EMRT_OK = 0,
  EMRT_ERR_INVALID_ARG = 1, /* bad pointer, size or parameter               */
  EMRT_ERR_OOM = 2,         /* device allocation failed                      */
  EMRT_ERR_CUDA = 3,        /* a CUDA runtime call failed                    */
  EMRT_ERR_CAPACITY = 4,    /* an output or scratch buffer was too small;
                               emrt_stats reports the required sizes         */
  EMRT_ERR_TIMEOUT = 5,     /* a bounded device wait gave up                 */
  EMRT_ERR_STATE = 6,       /* call order violated (e.g. trace before update) */
  EMRT_ERR_DEVICE = 7       /* kernel-raised error (traversal stack overflow,
                               a non-finite field) */
} emrt_status;

typedef struct emrt_scene_s *emrt_scene;

/* Static scene description.  All pointers are device pointers read during
 * emrt_scene_create only; the scene keeps its own copies. */
typedef struct {
  uint32_t n_static_faces;   /* F_s                                        */
  const uint32_t *face_off;  /* [F_s+1] vertex offsets into face_xyz       */
  const float *face_xyz;     /* [face_off[F_s]][3] polygon vertices         */
  const uint32_t *face_mat;  /* [F_s] material index                        */
  uint32_t n_tris;           /* T                                           */
  const float *tri_xyz;      /* [T][3][3]                                   */
  const uint32_t *tri_face;  /* [T] face of each triangle                   */
  uint32_t n_vehicles;       /* V (may be 0)                                */
  const float *veh_half;     /* [V][3] box half extents                     */
  uint32_t veh_mat;          /* material of every vehicle face              */
  uint32_t max_rx;           /* capacity for receivers                      */
  uint32_t max_tx;           /* capacity for transmitters (<= 255)          */
  uint32_t rebuild_every;    /* dynamic BVH: full rebuild every n updates,
                                refit otherwise (0 = default 1: on the city
                                a refitted tree cost more traversal than
                                the rebuild it saves)                       */
} emrt_scene_desc;

/* Sec. II-A/III-A: builds the static BVH once (binned SAH top-down on the
 * GPU, bottom-up boxes; a Morton-code LBVH if the SAH tree would be deeper
 * than the 64-entry traversal stack) and allocates the scene's buffers.
 * Synchronises the stream. */
emrt_status emrt_scene_create(const emrt_scene_desc *d, emrt_stream s,
                              emrt_scene *out);
void emrt_scene_destroy(emrt_scene sc);

/* Per-frame update (Sec. II-A dynamic BVH; Sec. III-C static base station,
 * tracked object speeds): vehicle boxes at veh_pos (box centres, [V][3]) with
 * velocities veh_vel; receivers rx_pos/rx_vel [n_rx][3]; transmitters
 * tx_pos/tx_vel [n_tx][3].  Refits the vehicle BVH (rebuilds it every
 * rebuild_every calls) and rebuilds the receiver BVH and the merged
 * vehicle + receiver BVH.  Trees of 4097-65536 primitives are built in one
 * cooperative launch whose blocks wait on one another at a bounded grid
 * barrier; a barrier that gives up makes the next emrt_sync return
 * EMRT_ERR_TIMEOUT (the trees are then invalid).  veh_* may be NULL when
 * V = 0; *_vel may be NULL for zero velocity. */
emrt_status emrt_scene_update_dynamic(emrt_scene sc, const float *veh_pos,
                                      const float *veh_vel, const float *rx_pos,
                                      const float *rx_vel, uint32_t n_rx,
                                      const float *tx_pos, const float *tx_vel,
                                      uint32_t n_tx, emrt_stream s);

typedef struct {
  uint32_t max_depth;   /* K reflections, 0..EMRT_MAX_DEPTH               */
  uint64_t n_rays;      /* N directions on the Fibonacci sphere per Tx      */
  uint64_t ray_offset;  /* traced subset: ray offset + stride * j, j<count  */
  uint64_t ray_stride;  /* >= 1                                            */
  uint64_t ray_count;   /* 0 = all rays from ray_offset                    */
  uint32_t flags;       /* EMRT_TRACE_*                                     */
} emrt_trace_params;

/* Caller-owned path set. */
typedef struct {
  uint32_t *rec;      /* [capacity][8] records (device)                    */
  uint32_t capacity;  /* records that rec can hold                          */
  uint32_t *count;    /* device uint32: records present / required          */
} emrt_paths;

/* Plain per-frame discovery (Sec. II-A): shoot-and-bounce from every Tx with
 * reception spheres r(L) = 1.25 sqrt(8 pi / (3 sqrt(3) N)) L, deduplicate
 * the face-ID sequences, accept them by the image method with occlusion
 * rays, write the accepted set to out in canonical order.  If more records
 * are needed than out->capacity, *out->count receives the required number,
 * the excess is dropped and emrt_sync returns EMRT_ERR_CAPACITY. */
emrt_status emrt_trace(emrt_scene sc, const emrt_trace_params *p,
                       emrt_paths *out, emrt_stream s);
/* With EMRT_TRACE_STATIC_CACHE (temporal coherence of the static geometry,
 * Sec. II-A/III-B: coherence between successive frames): every ray of the
 * ray set follows one specular chain, segment b of ray (tx, j) having a
 * static closest hit (t, face) that depends only on the transmitter position,
 * the direction and the static faces hit before.  The scene keeps that hit
 * per (bounce, tx, ray) -- 16 B each, (K+1) n_tx count entries, allocated with
 * the ray set's direction table -- tagged with an epoch of the transmitter's
 * position.  A later call reuses the entry of a segment whose chain hit only
 * static faces so far (then its origin, direction and excluded face are
 * those the entry was computed from) and still tests that segment against
 * the vehicles and the receivers of this frame; every other segment is
 * traced in full and, when its chain is still static, stored.  The output is
 * the output of the same call without the flag, bit for bit.  Forward
 * emrt_trace only (ignored by emrt_trace_backward and the batched form). */

/* Rediscovery into a path cache (Sec. II-A path caching, Sec. III-B): the
 * discovery and deduplication of emrt_trace with the ray set p, then
 * cache <- cache U (accepted candidates), where the candidates the cache
 * already holds are not validated again -- the cache must have been
 * revalidated (emrt_revalidate, compacting) with the current poses, so that
 * their acceptance is already known.  With EMRT_TRACE_REVALIDATE_FIRST the
 * call does that revalidation itself, on a side stream overlapping the
 * discovery (its own scratch, sized for the cache's capacity, allocated on
 * first use); the result is that of emrt_revalidate followed by this call.  The result equals emrt_trace into a
 * separate output followed by emrt_cache_merge, bit for bit (a candidate
 * held as a valid path lowers that record's smallest ray index, as the merge
 * would).  cache: canonical records (as the calls of this library write
 * them); it must have room for the union, else emrt_sync returns
 * EMRT_ERR_CAPACITY and the cache holds only its first capacity records.
 * EMRT_TRACE_KEEP_REJECTED is not accepted (EMRT_ERR_INVALID_ARG); the other
 * trace flags apply.  emrt_stats.accepted is the cache count after the
 * call. */
emrt_status emrt_rediscover(emrt_scene sc, const emrt_trace_params *p, emrt_paths *cache,
                            emrt_stream s);

/* Backward discovery (Sec. II-A: ray tracing from the receiver in the
 * visibility step): shoot-and-bounce from receivers, with the same Fibonacci
 * ray set p (per receiver instead of per Tx) and reception spheres of the
 * same radius r(L) around every transmitter.  Paths are reciprocal, so each
 * candidate is turned round -- transmitter first, face IDs in the order met
 * from the transmitter -- and then deduplicated, accepted and written exactly
 * as by emrt_trace (same record layout and canonical order; word 7 holds
 * the smallest backward ray index that found the path).
 * rx_ids: device uint32[n_ids] receiver indices to shoot from (distinct, each
 * < n_rx), or NULL for every receiver (n_ids ignored).  The ray ids pack
 * source << (32 - b) | ray index with b = bits(n_sources - 1), so the ray
 * count per receiver must be <= 2^(32 - b), and n_sources x count < 2^32;
 * otherwise EMRT_ERR_INVALID_ARG.  Capacity handling as emrt_trace. */
emrt_status emrt_trace_backward(emrt_scene sc, const emrt_trace_params *p,
                                const uint32_t *rx_ids, uint32_t n_ids,
                                emrt_paths *out, emrt_stream s);

/* The cached frame of emrt_revalidate without flags (invalid paths removed,
 * order kept); *n_evicted (device uint32, may be NULL) receives the number
 * of records removed. */
emrt_status emrt_revalidate_cache(emrt_scene sc, emrt_paths *cache, uint32_t *n_evicted,
                                  emrt_stream s);

/* Cached frame (Sec. II-A path caching, Sec. III-B): re-runs image-method
 * acceptance and occlusion on every record of `cache` with the current
 * poses; removes the paths that failed (keeps order) unless
 * EMRT_REVALIDATE_KEEP, in which case only EMRT_PATH_VALID is updated. */
emrt_status emrt_revalidate(emrt_scene sc, emrt_paths *cache, uint32_t flags,
                            emrt_stream s);

/* cache <- sorted union of cache and fresh, both in canonical order (as
 * emrt_trace, emrt_trace_backward, emrt_revalidate and emrt_cache_merge
 * write them): the two runs are merged, not re-sorted; an input out of order
 * makes the next emrt_sync return EMRT_ERR_INVALID_ARG.  Equal paths keep
 * the cache's record with the smaller ray index of the two. */
emrt_status emrt_cache_merge(emrt_scene sc, emrt_paths *cache,
                             const emrt_paths *fresh, emrt_stream s);

typedef struct {
  uint32_t n_mat;
  const double *eps_r;   /* [n_mat] relative permittivity (device)         */
  const double *sigma;   /* [n_mat] conductivity S/m (device)               */
  const double *gamma;   /* [n_mat] Table I coefficients, or NULL           */
  uint32_t const_gamma;  /* 1: Gamma_s = -gamma, Gamma_p = +gamma           */
} emrt_materials;

typedef struct {
  double *path_out;  /* [paths capacity][4]: Re a, Im a, tau (s), f_D (Hz);
                        a is the complex amplitude for 1 W transmit power  */
  double *pair_out;  /* [n_tx][n_rx][8]: Re h, Im h, sum|a|^2, mean f_D,
                        RMS Doppler spread, mean delay, RMS delay spread,
                        path count (h = coherent sum of a)                  */
  double *rx_out;    /* [n_rx][2]: received power (W) coherent per Tx and
                        summed over Tx; fully incoherent power (W)          */
} emrt_channel_out;

/* Field of every path in `paths` at frequency freq_hz (Sec. III-C, Eq. 3
 * generalised to moving endpoints and reflectors; Table III statistics).
 * Paths must be canonical (sorted).  Invalid arguments (null outputs,
 * freq_hz <= 0) return EMRT_ERR_INVALID_ARG; a non-finite result (e.g. NaN
 * material parameters) makes the next emrt_sync return EMRT_ERR_DEVICE. */
emrt_status emrt_channel(emrt_scene sc, const emrt_paths *paths,
                         const emrt_materials *m, double freq_hz,
                         double tx_power_w, emrt_channel_out *out,
                         emrt_stream s);

/* emrt_channel (Sec. III-C, Eq. 3 generalised; Table III statistics) at
 * n_freq frequencies (1..8) in one pass: outs[q] receives the results at
 * freq_hz[q] (host array), exactly as emrt_channel would (the frequencies
 * share each launch, one grid row per frequency).  outs[q].rx_out may be
 * NULL.  A non-finite result (e.g. NaN material parameters) makes the next
 * emrt_sync return EMRT_ERR_DEVICE; other errors as emrt_channel. */
emrt_status emrt_channel_multi(emrt_scene sc, const emrt_paths *paths, const emrt_materials *m,
                               const double *freq_hz, uint32_t n_freq, double tx_power_w,
                               emrt_channel_out *outs, emrt_stream s);

/* Adjoint of emrt_channel's coherent sums over a frozen path topology:
 * given dloss_dh [n_tx][n_rx][2] (d loss / d Re h, d loss / d Im h),
 * accumulates (overwrites) grad_eps [n_mat], grad_sigma [n_mat] and
 * grad_tx [n_tx][3].  Reflection points are recomputed, not stored.  A
 * non-finite amplitude or tangent (e.g. NaN material parameters) makes the
 * next emrt_sync return EMRT_ERR_DEVICE. */
emrt_status emrt_channel_backward(emrt_scene sc, const emrt_paths *paths,
                                  const emrt_materials *m, double freq_hz,
                                  const double *dloss_dh, double *grad_eps,
                                  double *grad_sigma, double *grad_tx,
                                  emrt_stream s);

/* Allocation-free variant of emrt_channel_backward, for callers that must
 * not allocate device memory after set-up: applications whose device memory
 * is owned by another allocator or capped (a cudaMalloc there can fail or
 * break the owner's accounting), and real-time loops that pre-allocate once
 * so that no call can stall in the allocator.  The paper has no counterpart;
 * it is a library service.
 *
 * Same arguments and results as emrt_channel_backward, but the per-path
 * tangent scratch lives in a fixed device array compiled into libemrt.so
 * (EMRT_NOALLOC_MAX_PATHS x 11 doubles, 5.8 MB, held by every GPU that loads
 * the library until the process exits) instead of scene-owned memory, and the
 * call allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine.  Requirements and behaviour:
 *  - paths->capacity must be <= EMRT_NOALLOC_MAX_PATHS, otherwise
 *    EMRT_ERR_INVALID_ARG is returned and nothing is launched;
 *  - the first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current and keeps it for the
 *    life of the process; make that first call before any stream capture
 *    begins.  cudaDeviceReset ends the library's use of that device (it also
 *    frees every scene there): the kept address is not looked up again;
 *  - every call on a device shares the one array: calls whose kernels overlap
 *    on the GPU (different streams without ordering) race and give wrong
 *    gradients; order them on one stream.  The array keeps the last call's
 *    contents; each call overwrites every entry it reads, so no clearing is
 *    needed;
 *  - a non-finite amplitude or tangent makes the next emrt_sync return
 *    EMRT_ERR_DEVICE, as for emrt_channel_backward. */
#define EMRT_NOALLOC_MAX_PATHS 65536u
emrt_status emrt_channel_backward_noalloc(emrt_scene sc, const emrt_paths *paths,
                                          const emrt_materials *m, double freq_hz,
                                          const double *dloss_dh, double *grad_eps,
                                          double *grad_sigma, double *grad_tx,
                                          emrt_stream s);

/* Channel correlation over a series of frames, Eq. 1 (Sec. III-B), read as
 * the normalised autocovariance of g(t) = |h(t)| (the printed denominator
 * E[g^2] E[g]^2 is dimensionally inconsistent):
 *   R(tau) = (mean_{t < F - tau} g(t) g(t + tau) - mu^2) / (mean_t g^2 - mu^2),
 * mu = mean_t g.  h: [n_frames][n_pairs][2] complex coherent sums (e.g. the
 * Re h, Im h of emrt_channel's pair_out gathered frame by frame); R:
 * [n_pairs][max_lag + 1].  Pairs whose |h| is constant get R = 0. */
emrt_status emrt_channel_correlation(const double *h, uint32_t n_frames, uint32_t n_pairs,
                                     uint32_t max_lag, double *R, emrt_stream s);

/* Coherence time per (tx, rx) from Eq. 2 (Sec. III-B) as printed:
 *   T_c = sqrt(1 / R^4 - 1) / (2 pi f_D theta^2)  [seconds],
 * R = r_threshold in (0, 1], f_D = freq |v_rx| / c the receiver's maximum
 * Doppler shift, theta the angle (radians) between the receiver's motion and
 * the direction from transmitter to receiver.  Infinite for a receiver at
 * rest or moving along that direction.  tc: [n_tx][n_rx]. */
emrt_status emrt_coherence_time(emrt_scene sc, double freq_hz, double r_threshold, double *tc,
                                emrt_stream s);

/* Per-receiver re-discovery schedule for cached frames.  Sec. III-A cuts a
 * receiver's trajectory into segments where spatial consistency is lost --
 * the LoS/NLoS condition or the position changes -- and reuses the channel
 * within a segment; Sec. III-B reuses cached paths within the coherence time
 * (Eq. 2).  Call once per frame after emrt_scene_update_dynamic.  Receiver r
 * is due for re-discovery when any of these holds:
 *   - it was never discovered (state[r][3] < 0);
 *   - the line of sight of some (tx, r) pair -- its direct path accepted by
 *     the image-method/occlusion test of emrt_trace, same margins -- differs
 *     from the one recorded at r's last discovery;
 *   - |p_r - state[r][0..2]|^2 >= d_seg^2 (FP64 from the float32 values);
 *   - the frames since r's last discovery, plus this one, reach
 *     min(max_interval, max(1, floor(T_c / dt_s))), T_c the smallest Eq. 2
 *     coherence time of r over the transmitters (emrt_coherence_time with
 *     freq_hz, r_threshold); dt_s = 0 leaves out T_c (interval max_interval).
 * A due receiver's state becomes (p_r, 0) and its LoS conditions are
 * recorded; another receiver's frame count (state[r][3]) advances by one.
 * state: device float [n_rx][4], caller-owned, start with w = -1;
 * los_ref: device uint8 [n_tx][n_rx], caller-owned (any initial value);
 * ids: device uint32 [n_rx] receives the due receivers in ascending order
 * and *n_due (device uint32) their number -- the list emrt_trace_backward
 * takes.  max_interval >= 1, dt_s >= 0, d_seg >= 0, freq_hz > 0 and
 * r_threshold in (0, 1], else EMRT_ERR_INVALID_ARG. */
emrt_status emrt_refresh_schedule(emrt_scene sc, float *state, uint8_t *los_ref, double freq_hz,
                                  double r_threshold, double dt_s, float d_seg,
                                  uint32_t max_interval, uint32_t *ids, uint32_t *n_due,
                                  emrt_stream s);

typedef struct {
  uint64_t segments[EMRT_MAX_DEPTH + 1]; /* closest-hit segments per bounce */
  uint64_t candidates;        /* reception-sphere detections                 */
  uint64_t unique_candidates; /* after deduplication                         */
  uint64_t accepted;          /* paths written                                */
  uint64_t occlusion_rays;    /* any-hit segments traced by acceptance (each
                                 leg as 4 pieces; pieces of a leg already
                                 found occluded are skipped, so the count
                                 varies a little from run to run)           */
  uint64_t node_visits;       /* static BVH inner nodes visited (closest hit) */
  uint64_t tri_tests;         /* triangles tested (closest hit)               */
  uint64_t dyn_node_visits;   /* vehicle BVH inner nodes visited              */
  uint64_t box_tests;         /* vehicle boxes tested                         */
  uint64_t rx_node_visits;    /* receiver BVH inner nodes visited             */
  uint64_t rx_tests;          /* receivers tested against a reception sphere  */
  uint32_t error_bits;        /* device error word                            */
  uint32_t required_candidates; /* scratch sizes needed by the last trace   */
  uint32_t required_paths;
  uint32_t pad;
  /* device time of the last emrt_trace (CUDA events on its stream), ms:
   * discovery stage (traversal kernels and ray sorts), deduplication,
   * image-method acceptance, whole call, and the closest-hit traversal
   * kernels alone (sum over bounces); a trace recorded into a caller's CUDA
   * graph and replayed from it leaves them at their last values */
  float traverse_ms, dedup_ms, accept_ms, trace_ms, bounce_ms;
  uint32_t pad2;
  uint64_t static_reused;     /* segments whose static closest hit came from
                                 the static-hit cache (EMRT_TRACE_STATIC_CACHE) */
  uint64_t deferred;          /* chains the cache walker could not finish
                                 from the cache (carried to their ends with
                                 the full static traversal)                  */
} emrt_stats;

/* Waits for the stream, reads and clears the device error word, returns the
 * first error recorded since the last emrt_sync and fills *st if non-NULL. */
emrt_status emrt_sync(emrt_scene sc, emrt_stream s, emrt_stats *st);

/* ---------------------------------------------------------------------
 * Batched discovery over many scenes of uneven size (the paper runs one
 * scene at a time).  Persistent traversal launches serve the rays of every
 * scene of the batch (depth-first: one launch carrying every chain to its
 * end, the untuned default; breadth-first: one launch per bounce);
 * deduplication, acceptance and the scatter to each scene's output follow
 * once.  The launch
 * sequence is captured into a CUDA graph on the first emrt_batch_trace and
 * replayed afterwards.  Limits: <= 64 scenes, <= 16 transmitters per scene,
 * <= 2^22 rays per transmitter. */
typedef struct emrt_batch_s *emrt_batch;

#define EMRT_BATCH_AUTOTUNE 0x1u /* time every traversal variant (form and
                                    block size; rays fetched per warp and
                                    coherence sort on or off for the
                                    breadth-first form) on this batch and keep
                                    the fastest;
                                    the choice is cached in the JSON file
                                    $EMRT_AUTOTUNE_CACHE (default
                                    $HOME/.emrt_autotune.json) and reused */
#define EMRT_BATCH_BREADTH_FIRST 0x2u /* without autotuning: the breadth-first
                                         form (one launch per bounce, ray
                                         sort) instead of the depth-first one;
                                         same records */

/* scenes[i] must have been updated (emrt_scene_update_dynamic) and keeps its
 * transmitter count for the life of the batch; params[i] and outs[i] are the
 * ray set and the caller-owned output of scene i (as for emrt_trace).  The
 * arrays are copied; the scenes and output buffers must outlive the batch.
 * Allocates the batch's scratch and direction tables; synchronises. */
emrt_status emrt_batch_create(const emrt_scene *scenes, uint32_t n,
                              const emrt_trace_params *params, emrt_paths *outs,
                              uint32_t flags, emrt_stream s, emrt_batch *out);
/* Discovery, deduplication and acceptance for every scene with the current
 * poses (the same result as emrt_trace on each scene).  Asynchronous; the
 * first call captures the graph.  After that first call, a call on a stream
 * that the caller is capturing into its own CUDA graph records the batch's
 * launch sequence into that graph instead (no host synchronisation; the
 * pinned per-scene table is copied by a node of the caller's graph, so the
 * scenes must keep their transmitter and receiver counts while the caller's
 * graph is replayed); calling it before the first uncaptured call returns
 * EMRT_ERR_STATE.  Begin such a capture after the batch's earlier calls have
 * completed (e.g. after emrt_batch_sync): the captured call rewrites the
 * pinned table without waiting for a copy still pending from them. */
emrt_status emrt_batch_trace(emrt_batch b, emrt_stream s);
/* Waits and reports errors as emrt_sync (stats summed over the batch). */
emrt_status emrt_batch_sync(emrt_batch b, emrt_stream s, emrt_stats *st);
/* One call for a batch: the first call with a given (scenes, params, outs)
 * creates the batch (emrt_batch_create, no autotuning) and captures its graph;
 * later calls with the same arrays replay it.  Traces, then synchronises the
 * stream and returns as emrt_batch_sync (the outputs' counts are written).
 * params and outs are arrays of n.  Destroying one of the scenes discards the
 * batches that use it. */
emrt_status emrt_trace_batched(const emrt_scene *scenes, uint32_t n,
                               const emrt_trace_params *params, emrt_paths *outs,
                               emrt_stream s);
/* Human-readable traversal variant chosen for the batch. */
emrt_status emrt_batch_config(emrt_batch b, char *buf, uint32_t len);
void emrt_batch_destroy(emrt_batch b);

const char *emrt_status_string(emrt_status e);

/* Number of kernel launches this library has issued in this process
 * (diagnostics; host-side counter). */
uint64_t emrt_kernel_launches(void);

/* Self-test of the bounded grid barrier that separates the phases of the
 * per-frame cooperative tree builds (no paper passage): one cooperative
 * launch of 4 blocks on the legacy default stream waits at the barrier for
 * 4 + missing_blocks arrivals, then the call synchronises the device.
 * *blocks_passed (host) = blocks that got through (4 when missing_blocks is
 * 0), *timed_out (host) = 1 when the blocks gave up after the barrier's
 * poll limit (about 0.7 s; always when missing_blocks > 0).  The
 * context stays usable.  EMRT_ERR_INVALID_ARG for null pointers or
 * missing_blocks > 1024, EMRT_ERR_CUDA if the launch fails. */
emrt_status emrt_selftest_grid_barrier(uint32_t missing_blocks, uint32_t *blocks_passed,
                                       uint32_t *timed_out);

#ifdef __cplusplus
}
#endif
#endif
