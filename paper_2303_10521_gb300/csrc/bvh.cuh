// LBVH construction and refit (Karras 2012 binary radix tree over 63-bit
// Morton codes; bottom-up box refit with per-node arrival counters).
#pragma once
#include "common.cuh"
#include "prims.cuh"

namespace emrt {

enum PrimKind { PRIM_TRI = 0, PRIM_BOX = 1, PRIM_POINT = 2 };

// Owned device buffers of one BVH.
struct BVHBuf {
  PrimKind kind = PRIM_TRI;
  uint32_t n = 0, cap = 0;
  float4 *nodes = nullptr;       // [cap-1][4]
  float4 *prims = nullptr;       // [cap][words per prim]
  uint32_t *leaf_parent = nullptr;  // [cap]  parent * 2 + side
  uint32_t *flags = nullptr;     // [cap]  refit arrival counters
  KeyW<2> *keys = nullptr, *keys2 = nullptr;  // [cap]
  uint32_t *idx = nullptr, *idx2 = nullptr;   // [cap]
  uint32_t *d_n = nullptr;       // device copy of n
  uint4 *nodes8 = nullptr;       // compressed 8-wide tree (static BVH), or null
  float4 *prims8 = nullptr;      // its triangles, in its own leaf order
  uint32_t n8 = 0;
  uint32_t leaf_bits = 0;        // see BVHView (2: multi-triangle SAH leaves)
  // Every leaf box is grown by `pad` metres on each side.  A box test takes a
  // plane's t as p idir - o idir, so the rounding of o idir shifts the plane
  // by up to 2^-24 |o| along its axis; the pad, 2^-21 times the largest
  // coordinate of the scene, keeps the test conservative for ray origins in
  // the scene (no cracks at box planes that are also triangle edges).
  float pad = 0.f;
  // scratch of the one-launch cooperative build (per-block digit counts and
  // the grid barrier), and the device error word it reports a barrier that
  // gave up to (ERR_WAIT; may be null)
  uint32_t *coop_hist = nullptr;
  uint32_t *coop_bar = nullptr;
  uint32_t *err_word = nullptr;
  BVHView view() const;
};

cudaError_t bvh_alloc(BVHBuf &b, PrimKind kind, uint32_t cap);
void bvh_free(BVHBuf &b);

// Scene bounding box used to quantise Morton codes: lo, hi (device float4[2]).
// Builds the hierarchy over n primitives given by `src`:
//   PRIM_TRI:   src = float[n][9] triangle vertices, ids = face id per triangle
//   PRIM_BOX:   src = float4 lo[n], hi[n] (interleaved pairs), ids = vehicle id
//   PRIM_POINT: src = float4[n] positions, ids = point id
// After build the prims are in leaf order and boxes are refitted.
cudaError_t bvh_build_tris(BVHBuf &b, const float *tri_xyz, const uint32_t *tri_face,
                           uint32_t n, const float4 *bbox, uint32_t *hist, cudaStream_t s);
cudaError_t bvh_build_boxes(BVHBuf &b, const float4 *lo, const float4 *hi, uint32_t n,
                            const float4 *bbox, uint32_t *hist, cudaStream_t s);
cudaError_t bvh_build_points(BVHBuf &b, const float4 *pts, uint32_t n, const float4 *bbox,
                             uint32_t *hist, cudaStream_t s);
// Top-down binned-SAH build of a triangle BVH (same node format as the
// LBVH; used for the static geometry, which is built once).  Two
// consecutive triangles of one face with the same bounding box (the halves
// of a planar quad) share one leaf; other leaves hold one triangle.
// Synchronises.
cudaError_t bvh_build_tris_sah(BVHBuf &b, const float *tri_xyz, const uint32_t *tri_face,
                               uint32_t n, cudaStream_t s);
// Moves box primitives to new corners (vehicle id kept in lo.w) and refits.
cudaError_t bvh_refit_boxes(BVHBuf &b, const float4 *lo, const float4 *hi, cudaStream_t s);

// Builds the compressed 8-wide tree of a triangle BVH b (built, refitted)
// into b.nodes8 / b.prims8 (layout in BVHView): every wide node takes its
// binary node's two children and repeatedly opens the inner child of largest
// surface area until it holds 8 children; child boxes are quantised to 8 bits
// on the node's grid.  Synchronises the stream (build time only).
cudaError_t bvh8_build(BVHBuf &b, cudaStream_t s);

// Runs the per-frame builds' grid barrier once in a cooperative launch of 4
// blocks expecting 4 + missing arrivals (synchronous): passed = blocks that
// got through, timed_out = 1 when a block gave up (ERR_WAIT).
cudaError_t grid_barrier_selftest(uint32_t missing, uint32_t *passed, uint32_t *timed_out);

// Axis-aligned bounds of n float[9] triangles, written to bbox[2].
void bbox_of_tris(const float *tri_xyz, uint32_t n, float4 *bbox, cudaStream_t s);

}  // namespace emrt
