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
  float4 *nodes4 = nullptr;      // 4-wide collapse (static BVH), or null
  uint32_t n4 = 0;
  uint32_t leaf_bits = 0;        // see BVHView (2: multi-triangle SAH leaves)
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
// LBVH; used for the static geometry, which is built once).  Synchronises.
cudaError_t bvh_build_tris_sah(BVHBuf &b, const float *tri_xyz, const uint32_t *tri_face,
                               uint32_t n, cudaStream_t s);
// Moves box primitives to new corners (vehicle id kept in lo.w) and refits.
cudaError_t bvh_refit_boxes(BVHBuf &b, const float4 *lo, const float4 *hi, cudaStream_t s);

// Collapses the binary tree of b (built, refitted) into 4-wide nodes
// (b.nodes4): every 4-wide node takes its binary node's two children and
// repeatedly opens the inner child of largest surface area until it holds 4
// children.  Synchronises the stream (build time only).
cudaError_t bvh4_collapse(BVHBuf &b, cudaStream_t s);

// Axis-aligned bounds of n float[9] triangles, written to bbox[2].
void bbox_of_tris(const float *tri_xyz, uint32_t n, float4 *bbox, cudaStream_t s);

}  // namespace emrt
