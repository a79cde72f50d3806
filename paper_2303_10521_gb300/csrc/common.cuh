// Shared device-side definitions of the emrt CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "emrt.h"

namespace emrt {

// ---------------------------------------------------------------------------
// device error word bits (read and cleared by emrt_sync)
enum : uint32_t {
  ERR_CAND_OVERFLOW = 1u,   // candidate scratch too small
  ERR_PATH_OVERFLOW = 2u,   // caller's path buffer too small
  ERR_STACK = 4u,           // traversal stack overflow
  ERR_RAY_OVERFLOW = 8u,    // ray scratch too small (internal bug)
  ERR_UNSORTED = 16u,       // a merge input is not in canonical order
  ERR_WAIT = 64u,           // a bounded wait between blocks gave up
};

// per-call counters kept in device memory (one struct per scene)
struct Counters {
  uint32_t err;                            // error bits (cleared by emrt_sync)
  uint32_t n_ray[EMRT_MAX_DEPTH + 2];      // rays entering bounce b (b >= 1)
  uint32_t work[EMRT_MAX_DEPTH + 1];       // persistent-kernel work cursors
  uint32_t n_cand;                         // candidates appended (may exceed capacity)
  uint32_t n_eff;                          // candidates stored
  uint32_t n_unique;
  uint32_t n_accepted;
  uint32_t tmp;
  uint32_t chain_work;                     // work cursor of the cache walker
  unsigned long long segments[EMRT_MAX_DEPTH + 1];
  unsigned long long node_visits;     // static BVH inner nodes visited
  unsigned long long tri_tests;       // triangles tested
  unsigned long long dyn_node_visits; // vehicle BVH inner nodes visited
  unsigned long long box_tests;       // vehicle boxes tested
  unsigned long long rx_node_visits;  // receiver BVH inner nodes visited
  unsigned long long rx_tests;        // receivers tested against a sphere
  unsigned long long occl_rays;
  unsigned long long static_reused;   // static hits taken from the cache
  unsigned long long deferred;        // chains the cache walker queued
};

// ---------------------------------------------------------------------------
// BVH (binary LBVH, Karras 2012) device view.
// Node i occupies 4 float4 (64 B):
//   [0] c0.lo.x c0.hi.x c0.lo.y c0.hi.y
//   [1] c1.lo.x c1.hi.x c1.lo.y c1.hi.y
//   [2] c0.lo.z c0.hi.z c1.lo.z c1.hi.z
//   [3] (int) c0, c1, parent, 0     child >= 0: inner node, < 0: leaf ~prim
struct BVHView {
  const uint4 *nodes8;   // optional compressed 8-wide tree of a triangle BVH
                         // (5 uint4 per node: origin, exponents and inner
                         // mask; first child, leaf mask, first triangle,
                         // leaf meta; 8-bit child boxes along x, y, z)
  const float4 *prims8;  // its triangles (3 float4 each, as prims)
  const float4 *nodes;
  const float4 *prims;  // triangles: 3 float4 (v0 with face id bits in .w,
                        // v1, v2); boxes: 2 float4 (lo with vehicle id bits in
                        // .w, hi); points: 1 float4 (xyz, receiver id bits)
  int root;             // 0 (inner), ~0 (single leaf)
  uint32_t n_prims;     // 0 = empty
  uint32_t leaf_bits;   // leaf code ~c: c = first prim (0), or first << 2 |
                        // (count - 1) for leaves of 1-4 prims (2); ~0 is
                        // prim 0 alone either way
};

// Index of the path this thread takes among the block's records base ..
// base + blockDim.x - 1 (8 words each), handed out in order of depth (word
// 2, low 4 bits; depths above EMRT_MAX_DEPTH and records past cnt last), so
// that a warp's paths mostly share their number of reflections and its
// per-bounce loops run for its own depth.  A result >= cnt means none.
// Called by every thread of the block (it synchronises); s_cnt holds
// EMRT_MAX_DEPTH + 2 words, s_order blockDim.x.
__device__ inline uint32_t depth_ordered(const uint32_t *rec, uint32_t base, uint32_t cnt,
                                         uint32_t *s_cnt, uint32_t *s_order) {
  if (threadIdx.x <= EMRT_MAX_DEPTH + 1) s_cnt[threadIdx.x] = 0u;
  __syncthreads();
  const uint32_t mine = base + threadIdx.x;
  const uint32_t bucket =
      mine < cnt ? min(rec[8ull * mine + 2] & 15u, (uint32_t)EMRT_MAX_DEPTH + 1u) : EMRT_MAX_DEPTH + 1u;
  const uint32_t rank = atomicAdd(&s_cnt[bucket], 1u);
  __syncthreads();
  uint32_t start = 0;
  for (uint32_t q = 0; q < bucket; q++) start += s_cnt[q];
  s_order[start + rank] = mine;
  __syncthreads();
  const uint32_t i = s_order[threadIdx.x];
  __syncthreads();
  return i;
}

// ray state between bounces: 48 B
struct Ray {
  float4 o_L;    // origin, unfolded length travelled so far (L_acc)
  float4 d_id;   // unit direction, (tx << 24 | ray index j) bits
  uint4 faces;   // face IDs of the reflections so far
};

struct Vec3 { float x, y, z; };

__host__ __device__ inline float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ inline float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ inline float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ inline float3 operator*(float3 a, float s) { return make_float3(a.x * s, a.y * s, a.z * s); }
__device__ inline float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

struct D3 { double x, y, z; };
__device__ inline D3 mkd(double x, double y, double z) { D3 r; r.x = x; r.y = y; r.z = z; return r; }
__device__ inline D3 operator+(D3 a, D3 b) { return mkd(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ inline D3 operator-(D3 a, D3 b) { return mkd(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ inline D3 operator*(D3 a, double s) { return mkd(a.x * s, a.y * s, a.z * s); }
__device__ inline double dotd(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ inline D3 crossd(D3 a, D3 b) {
  return mkd(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ inline double normd(D3 a) { return sqrt(dotd(a, a)); }
__device__ inline D3 tod(float3 a) { return mkd(a.x, a.y, a.z); }

__device__ inline uint32_t lanemask_lt() {
  uint32_t m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Warp-aggregated append: every active lane that calls this gets a distinct
// slot; one atomicAdd per converged group of lanes.
__device__ inline uint32_t warp_append(uint32_t *counter) {
  uint32_t m = __activemask();
  uint32_t lane = threadIdx.x & 31;
  uint32_t leader = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(counter, (uint32_t)__popc(m));
  base = __shfl_sync(m, base, leader);
  return base + __popc(m & lanemask_lt());
}

// Warp-aggregated append to one of several counters: every active lane gets
// a distinct slot of counters[key]; lanes are grouped by key first, one
// atomicAdd per group.
__device__ inline uint32_t warp_append_keyed(uint32_t *counters, uint32_t key) {
  uint32_t m = __activemask();
  uint32_t grp = __match_any_sync(m, key);
  uint32_t lane = threadIdx.x & 31;
  uint32_t leader = __ffs(grp) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(counters + key, (uint32_t)__popc(grp));
  base = __shfl_sync(grp, base, leader);
  return base + __popc(grp & lanemask_lt());
}

// scene geometry (device views) shared by trace, acceptance and field
struct GeomView {
  BVHView stat;            // static triangles
  BVHView dyn;             // vehicle boxes
  BVHView rxb;             // receiver points
  BVHView mix;             // vehicles and receivers in one tree (or empty):
                           // prims 0..n_veh-1 boxes, then receiver points
  const double4_32a *face_plane;  // [F_s] unit normal, offset
  const uint4 *face_info;     // [F_s] vertex offset, vertex count, material, 0
  const float4 *face_vert;    // [NV] polygon vertices
  const float4 *veh_lo;       // [V] box corners (w unused)
  const float4 *veh_hi;
  const float4 *veh_vel;      // [V]
  const float4 *rx_pos;       // [R]
  const float4 *rx_vel;
  const float4 *tx_pos;       // [X]
  const float4 *tx_vel;
  uint32_t n_static_faces, n_veh, n_rx, n_tx, veh_mat;
};

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// host-side count of kernel launches issued by this library (diagnostics)
void note_launch();
unsigned long long launch_count();

}  // namespace emrt
