// LBVH build and refit.  Binary radix tree of Karras (2012, "Maximizing
// parallelism in the construction of BVHs, octrees and k-d trees"), restated
// from the published algorithm; boxes are filled bottom-up with one arrival
// counter per inner node (the second thread to arrive merges the children).
#include <cfloat>

#include <cuda/atomic>

#include "bvh.cuh"

namespace emrt {

namespace {

__device__ inline uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | x << 32) & 0x1f00000000ffffull;
  x = (x | x << 16) & 0x1f0000ff0000ffull;
  x = (x | x << 8) & 0x100f00f00f00f00full;
  x = (x | x << 4) & 0x10c30c30c30c30c3ull;
  x = (x | x << 2) & 0x1249249249249249ull;
  return x;
}

// Morton code (3 AB bits, AB <= 21 per axis) of p quantised in the cube
// spanned by the largest extent of the box (all axes share one scale), so
// that a flat scene is split along its long axes first instead of slicing it
// into thin horizontal slabs.  Equal codes are told apart by index in the
// hierarchy (delta), so coarse codes only cost tree quality.
template <int AB>
__device__ inline uint64_t morton_code(float3 p, const float4 *bb) {
  float4 lo = bb[0], hi = bb[1];
  float ext = fmaxf(fmaxf(hi.x - lo.x, hi.y - lo.y), fmaxf(hi.z - lo.z, 1e-6f));
  float q[3] = {(p.x - lo.x) / ext, (p.y - lo.y) / ext, (p.z - lo.z) / ext};
  uint32_t c[3];
  for (int k = 0; k < 3; k++)
    c[k] = (uint32_t)(fminf(fmaxf(q[k], 0.f), 1.f) * (float)((1u << AB) - 1u));
  return spread3(c[0]) << 2 | spread3(c[1]) << 1 | spread3(c[2]);
}
// code bits per primitive kind: the static triangles (LBVH fallback) use 63;
// vehicle boxes and receiver points, rebuilt every frame, use 30 (2 m cells
// over a 2 km cube) so that their sort takes four passes instead of eight
constexpr int kMortonBitsTri = 21, kMortonBitsDyn = 10;

__device__ inline void put_key(KeyW<2> &k, uint64_t v) {
  k.w[0] = (uint32_t)v;
  k.w[1] = (uint32_t)(v >> 32);
}
__device__ inline uint64_t get_key(const KeyW<2> &k) {
  return (uint64_t)k.w[1] << 32 | k.w[0];
}

__global__ void k_morton_tris(const float *t, uint32_t n, const float4 *bb, KeyW<2> *keys,
                              uint32_t *idx) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float *v = t + 9ull * i;
  float3 c = make_float3((v[0] + v[3] + v[6]) * (1.f / 3.f), (v[1] + v[4] + v[7]) * (1.f / 3.f),
                         (v[2] + v[5] + v[8]) * (1.f / 3.f));
  put_key(keys[i], morton_code<kMortonBitsTri>(c, bb));
  idx[i] = i;
}

__global__ void k_morton_boxes(const float4 *lo, const float4 *hi, uint32_t n, const float4 *bb,
                               KeyW<2> *keys, uint32_t *idx) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 a = lo[i], b = hi[i];
  put_key(keys[i], morton_code<kMortonBitsDyn>(
                       make_float3(0.5f * (a.x + b.x), 0.5f * (a.y + b.y), 0.5f * (a.z + b.z)), bb));
  idx[i] = i;
}

__global__ void k_morton_points(const float4 *p, uint32_t n, const float4 *bb, KeyW<2> *keys,
                                uint32_t *idx) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  put_key(keys[i], morton_code<kMortonBitsDyn>(f3(p[i]), bb));
  idx[i] = i;
}

// Inner node i in [0, n-2] of the radix tree over the sorted keys k: its
// range, split and children, and the parent links of the children.
template <typename KeyAt>
__device__ inline void hierarchy_node(KeyAt key, int n, int i, float4 *nodes,
                                      uint32_t *leaf_parent) {
  auto delta = [&](int a, int c) -> int {
    if (c < 0 || c >= n) return -1;
    const uint64_t x = key(a), y = key(c);
    if (x == y) return 64 + __clz(a ^ c);
    return __clzll(x ^ y);
  };
  int d = (delta(i, i + 1) - delta(i, i - 1)) >= 0 ? 1 : -1;
  int dmin = delta(i, i - d);
  int lmax = 2;
  while (delta(i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(i, i + (l + t) * d) > dmin) l += t;
  int j = i + l * d;
  int dnode = delta(i, j);
  int s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (delta(i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  int gamma = i + s * d + min(d, 0);
  int left = min(i, j) == gamma ? ~gamma : gamma;
  int right = max(i, j) == gamma + 1 ? ~(gamma + 1) : gamma + 1;
  int *n3 = reinterpret_cast<int *>(nodes + 4ll * i + 3);
  n3[0] = left;
  n3[1] = right;
  n3[3] = 0;
  int code0 = 2 * i, code1 = 2 * i + 1;
  if (left < 0) leaf_parent[~left] = code0;
  else reinterpret_cast<int *>(nodes + 4ll * left + 3)[2] = code0;
  if (right < 0) leaf_parent[~right] = code1;
  else reinterpret_cast<int *>(nodes + 4ll * right + 3)[2] = code1;
  if (i == 0) n3[2] = -1;
}

// one thread per inner node i in [0, n-2]
__global__ void k_hierarchy(const KeyW<2> *k, int n, float4 *nodes, uint32_t *leaf_parent) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  hierarchy_node([k](int a) { return get_key(k[a]); }, n, i, nodes, leaf_parent);
}

__global__ void k_gather_tris(const float *t, const uint32_t *face, const uint32_t *idx,
                              uint32_t n, float4 *prims) {
  uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  uint32_t s = idx[g];
  const float *v = t + 9ull * s;
  prims[3ull * g + 0] = make_float4(v[0], v[1], v[2], __uint_as_float(face[s]));
  prims[3ull * g + 1] = make_float4(v[3], v[4], v[5], 0.f);
  prims[3ull * g + 2] = make_float4(v[6], v[7], v[8], 0.f);
}

__global__ void k_gather_boxes(const float4 *lo, const float4 *hi, const uint32_t *idx, uint32_t n,
                               float4 *prims) {
  uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  uint32_t s = idx[g];
  float4 a = lo[s], b = hi[s];
  prims[2ull * g + 0] = make_float4(a.x, a.y, a.z, __uint_as_float(s));
  prims[2ull * g + 1] = make_float4(b.x, b.y, b.z, 0.f);
}

__global__ void k_move_boxes(const float4 *lo, const float4 *hi, uint32_t n, float4 *prims) {
  uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  uint32_t s = __float_as_uint(prims[2ull * g].w);
  float4 a = lo[s], b = hi[s];
  prims[2ull * g + 0] = make_float4(a.x, a.y, a.z, __uint_as_float(s));
  prims[2ull * g + 1] = make_float4(b.x, b.y, b.z, 0.f);
}

__global__ void k_gather_points(const float4 *p, const uint32_t *idx, uint32_t n, float4 *prims) {
  uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  uint32_t s = idx[g];
  float4 a = p[s];
  prims[g] = make_float4(a.x, a.y, a.z, __uint_as_float(s));
}

struct Box { float3 lo, hi; };

template <int KIND>
__device__ inline Box prim_box(const float4 *prims, uint32_t g) {
  Box b;
  if (KIND == PRIM_TRI) {
    float3 a = f3(prims[3ull * g]), c = f3(prims[3ull * g + 1]), d = f3(prims[3ull * g + 2]);
    b.lo = make_float3(fminf(a.x, fminf(c.x, d.x)), fminf(a.y, fminf(c.y, d.y)), fminf(a.z, fminf(c.z, d.z)));
    b.hi = make_float3(fmaxf(a.x, fmaxf(c.x, d.x)), fmaxf(a.y, fmaxf(c.y, d.y)), fmaxf(a.z, fmaxf(c.z, d.z)));
  } else if (KIND == PRIM_BOX) {
    b.lo = f3(prims[2ull * g]);
    b.hi = f3(prims[2ull * g + 1]);
  } else {
    b.lo = b.hi = f3(prims[g]);
  }
  return b;
}

// From a child box b whose parent link is `code` (parent * 2 + side) towards
// the root: the box is written into its parent, and the second thread to
// arrive at a node (arrival counters `flags`, global or shared) continues
// with the node's own box.  The arrival is one acquire-release atomic: it
// publishes this thread's box and, for the second arrival, makes the
// sibling's visible (no full fences; each level is on the critical path).
__device__ inline void refit_up(Box b, int code, float4 *nodes, uint32_t *flags) {
  for (int guard = 0; guard < 4096; guard++) {  // tree depth bound (safety net)
    const int p = code >> 1, side = code & 1;
    float4 *np = nodes + 4ll * p;
    reinterpret_cast<float4 *>(np + side)[0] = make_float4(b.lo.x, b.hi.x, b.lo.y, b.hi.y);
    reinterpret_cast<float2 *>(np + 2)[side] = make_float2(b.lo.z, b.hi.z);
    cuda::atomic_ref<uint32_t, cuda::thread_scope_device> arrivals(flags[p]);
    if (arrivals.fetch_add(1u, cuda::memory_order_acq_rel) == 0) return;
    const float4 a0 = __ldcg(np), a1 = __ldcg(np + 1), a2 = __ldcg(np + 2);
    b.lo = make_float3(fminf(a0.x, a1.x), fminf(a0.z, a1.z), fminf(a2.x, a2.z));
    b.hi = make_float3(fmaxf(a0.y, a1.y), fmaxf(a0.w, a1.w), fmaxf(a2.y, a2.w));
    const int pc = __ldcg(reinterpret_cast<const int *>(np + 3) + 2);
    if (pc < 0) return;
    code = pc;
  }
}

// Bottom-up boxes: one thread per leaf walks to the root; the second child
// to arrive at a node continues.  MULTI: leaves of 1-4 prims (leaf code
// ~(first << 2 | count - 1)); prims other than a leaf's first have
// leaf_parent 0xFFFFFFFF.
template <int KIND, bool MULTI = false>
__global__ void k_refit(const float4 *prims, uint32_t n, float4 *nodes, const uint32_t *leaf_parent,
                        uint32_t *flags, float pad) {
  uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n || n < 2) return;
  if (MULTI && leaf_parent[g] == 0xffffffffu) return;
  Box b = prim_box<KIND>(prims, g);
  int code = (int)leaf_parent[g];
  if (MULTI) {
    const int lc = reinterpret_cast<const int *>(nodes + 4ll * (code >> 1) + 3)[code & 1];
    const uint32_t cnt = ((uint32_t)(~lc) & 3u) + 1u;
    for (uint32_t q = 1; q < cnt && g + q < n; q++) {
      Box c = prim_box<KIND>(prims, g + q);
      b.lo = make_float3(fminf(b.lo.x, c.lo.x), fminf(b.lo.y, c.lo.y), fminf(b.lo.z, c.lo.z));
      b.hi = make_float3(fmaxf(b.hi.x, c.hi.x), fmaxf(b.hi.y, c.hi.y), fmaxf(b.hi.z, c.hi.z));
    }
  }
  b.lo = make_float3(b.lo.x - pad, b.lo.y - pad, b.lo.z - pad);
  b.hi = make_float3(b.hi.x + pad, b.hi.y + pad, b.hi.z + pad);
  refit_up(b, code, nodes, flags);
}

struct Child {
  int code;
  float lo[3], hi[3];
};

__device__ inline Child child_of(const float4 *nodes, int p, int side) {
  const float4 *np = nodes + 4ll * p;
  float4 a = np[side], z = np[2];
  Child c;
  c.code = reinterpret_cast<const int *>(np + 3)[side];
  c.lo[0] = a.x; c.hi[0] = a.y; c.lo[1] = a.z; c.hi[1] = a.w;
  c.lo[2] = side ? z.z : z.x;
  c.hi[2] = side ? z.w : z.y;
  return c;
}

__device__ inline float half_area(const Child &c) {
  float dx = c.hi[0] - c.lo[0], dy = c.hi[1] - c.lo[1], dz = c.hi[2] - c.lo[2];
  return dx * dy + dy * dz + dz * dx;
}

// ---------------------------------------------------------------------------
// Compressed 8-wide BVH: the quantised wide-BVH family of Ylitie, Karras and
// Laine (HPG 2017), restated.  A node holds up to 8 children of the binary
// tree (the inner child of largest surface area is opened until 8 are
// gathered); their boxes are 8-bit offsets on a per-node grid -- origin P,
// a power-of-two quantum per axis -- so a node is 80 B for 8 child boxes
// where the binary tree spends 64 B on 2.  Children are placed in the 8
// slots so that a ray whose direction has sign pattern o (bit a set when
// axis a is negative) meets them roughly near to far when it visits slots
// o ^ 0, o ^ 1, ..., o ^ 7: slot s receives, greedily, the child with the
// smallest offset from the node centre along the diagonal of sign pattern s.
// Node layout (5 x uint4):
//   [0] P.x, P.y, P.z (float bits), e_x | e_y << 8 | e_z << 16 | imask << 24
//       (e: biased exponent of the quantum, 2^(e - 127); imask: inner slots)
//   [1] first child node | lmask << 24 (leaf slots), first triangle,
//       leaf meta of slots 0-3 and 4-7 (byte: offset | (count - 1) << 5)
//   [2] x: low bytes of slots 0-3, 4-7, high bytes of slots 0-3, 4-7
//   [3] y, [4] z, as [2]
// Inner children of a node are consecutive nodes in slot order; the
// triangles of its leaf children are consecutive in the wide tree's own
// triangle array.  Every quantised box contains its child's box grown by two
// quanta (and the quantum is at least one float ulp of the node's
// coordinates), which covers the rounding of the traversal's decode.
constexpr int kWideQuantPad = 2;

__device__ inline float wide_ulp(float a) {
  const float m = fabsf(a);
  return m > 0.f ? nextafterf(m, 3.4e38f) - m : 1.17549435e-38f;
}

// Quantises one axis of up to 8 child boxes on the node's grid: returns the
// biased exponent and the origin; q_lo/q_hi receive the grid coordinates.
__device__ inline uint32_t wide_axis(const float *clo, const float *chi, int cnt, float lo, float hi,
                                     float &P, uint8_t *q_lo, uint8_t *q_hi) {
  const double ext = (double)hi - (double)lo;
  const float u = fmaxf(wide_ulp(lo), wide_ulp(hi));
  int e = ilogb(u);  // the quantum is at least one ulp of the coordinates
  while (e < 127 && ldexp(1.0, e) * (255.0 - 2.0 * kWideQuantPad - 1.0) < ext) e++;
  for (;; e++) {
    const double q = ldexp(1.0, e);
    P = (float)((double)lo - kWideQuantPad * q);
    bool ok = true;
    for (int k = 0; k < cnt && ok; k++) {
      const double a = floor(((double)clo[k] - (double)P) / q) - kWideQuantPad;
      const double b = ceil(((double)chi[k] - (double)P) / q) + kWideQuantPad;
      if (b > 255.0 || b < 0.0) { ok = false; break; }
      q_lo[k] = (uint8_t)(a < 0.0 ? 0.0 : a);
      q_hi[k] = (uint8_t)b;
    }
    if (ok || e >= 127) return (uint32_t)(e + 127);  // e >= 127: degenerate input
  }
}

// one thread per wide node of the current level
__global__ void k_wide8(const float4 *bn, const float4 *bprims, uint32_t leaf_bits,
                        const uint32_t *in_bin, const uint32_t *in_dst, const uint32_t *n_in,
                        uint4 *out8, float4 *tris8, uint32_t *out_bin, uint32_t *out_dst,
                        uint32_t *n_out, uint32_t *n_alloc, uint32_t *t_alloc) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *n_in) return;
  const int b = (int)in_bin[i];
  const uint32_t dst = in_dst[i];
  Child c[8];
  int cnt = 2;
  c[0] = child_of(bn, b, 0);
  c[1] = child_of(bn, b, 1);
  while (cnt < 8) {
    int best = -1;
    float ba = -1.f;
    for (int k = 0; k < cnt; k++)
      if (c[k].code >= 0 && half_area(c[k]) > ba) {
        ba = half_area(c[k]);
        best = k;
      }
    if (best < 0) break;
    const int nb = c[best].code;
    c[best] = child_of(bn, nb, 0);
    c[cnt++] = child_of(bn, nb, 1);
  }
  float lo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, hi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
  for (int k = 0; k < cnt; k++)
    for (int a = 0; a < 3; a++) {
      lo[a] = fminf(lo[a], c[k].lo[a]);
      hi[a] = fmaxf(hi[a], c[k].hi[a]);
    }
  // slots: greedily the (slot, child) pair of smallest offset along the
  // slot's diagonal
  int in_slot[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
  uint32_t used_child = 0;
  for (int round = 0; round < cnt; round++) {
    float bc = 3.4e38f;
    int bs = -1, bk = -1;
    for (int sl = 0; sl < 8; sl++) {
      if (in_slot[sl] >= 0) continue;
      for (int k = 0; k < cnt; k++) {
        if (used_child >> k & 1u) continue;
        float d = 0.f;
        for (int a = 0; a < 3; a++) {
          const float off = (c[k].lo[a] + c[k].hi[a]) - (lo[a] + hi[a]);
          d += (sl >> a & 1) ? -off : off;
        }
        if (d < bc) { bc = d; bs = sl; bk = k; }
      }
    }
    in_slot[bs] = bk;
    used_child |= 1u << bk;
  }
  uint32_t n_inner = 0, n_tris = 0;
  for (int k = 0; k < cnt; k++) {
    if (c[k].code >= 0) {
      n_inner++;
    } else {
      const uint32_t lc = (uint32_t)(~c[k].code);
      n_tris += leaf_bits ? (lc & 3u) + 1u : 1u;
    }
  }
  const uint32_t child_base = n_inner ? atomicAdd(n_alloc, n_inner) : 0u;
  const uint32_t tri_base = n_tris ? atomicAdd(t_alloc, n_tris) : 0u;
  uint32_t imask = 0, lmask = 0, meta[2] = {0u, 0u}, rank = 0, off = 0;
  float clo[3][8], chi[3][8];
  int ord = 0;
  for (int sl = 0; sl < 8; sl++) {
    const int k = in_slot[sl];
    if (k < 0) continue;
    for (int a = 0; a < 3; a++) {
      clo[a][ord] = c[k].lo[a];
      chi[a][ord] = c[k].hi[a];
    }
    ord++;
    if (c[k].code >= 0) {
      imask |= 1u << sl;
      const uint32_t q = atomicAdd(n_out, 1u);
      out_bin[q] = (uint32_t)c[k].code;
      out_dst[q] = child_base + rank++;
    } else {
      const uint32_t lc = (uint32_t)(~c[k].code);
      const uint32_t first = leaf_bits ? lc >> 2 : lc, n = leaf_bits ? (lc & 3u) + 1u : 1u;
      for (uint32_t t = 0; t < n; t++)
        for (int w = 0; w < 3; w++)
          tris8[3ull * (tri_base + off + t) + w] = bprims[3ull * (first + t) + w];
      lmask |= 1u << sl;
      meta[sl >> 2] |= (off | (n - 1u) << 5) << (8 * (sl & 3));
      off += n;
    }
  }
  uint8_t qlo[3][8] = {}, qhi[3][8] = {};
  float P[3];
  uint32_t ex[3];
  for (int a = 0; a < 3; a++) ex[a] = wide_axis(clo[a], chi[a], cnt, lo[a], hi[a], P[a], qlo[a], qhi[a]);
  // bytes back from child order to slot order
  uint32_t w[3][4] = {};
  ord = 0;
  for (int sl = 0; sl < 8; sl++) {
    if (in_slot[sl] < 0) continue;
    for (int a = 0; a < 3; a++) {
      w[a][sl >> 2] |= (uint32_t)qlo[a][ord] << (8 * (sl & 3));
      w[a][2 + (sl >> 2)] |= (uint32_t)qhi[a][ord] << (8 * (sl & 3));
    }
    ord++;
  }
  uint4 *o = out8 + 5ull * dst;
  o[0] = make_uint4(__float_as_uint(P[0]), __float_as_uint(P[1]), __float_as_uint(P[2]),
                    ex[0] | ex[1] << 8 | ex[2] << 16 | imask << 24);
  o[1] = make_uint4(child_base | lmask << 24, tri_base, meta[0], meta[1]);
  for (int a = 0; a < 3; a++) o[2 + a] = make_uint4(w[a][0], w[a][1], w[a][2], w[a][3]);
}

__device__ inline uint32_t f2o(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ inline float o2f(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void k_bbox_init(uint32_t *acc) {
  if (threadIdx.x < 3) acc[threadIdx.x] = 0xffffffffu;
  else if (threadIdx.x < 6) acc[threadIdx.x] = 0u;
}

__global__ void k_bbox_tris(const float *t, uint32_t n, uint32_t *acc) {
  float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += gridDim.x * blockDim.x) {
    const float *v = t + 3ull * i;
    for (int k = 0; k < 3; k++) {
      lo[k] = fminf(lo[k], v[k]);
      hi[k] = fmaxf(hi[k], v[k]);
    }
  }
  for (int k = 0; k < 3; k++) {
    for (int o = 16; o; o >>= 1) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&acc[k], f2o(lo[k]));
      atomicMax(&acc[3 + k], f2o(hi[k]));
    }
  }
}

__global__ void k_bbox_fin(const uint32_t *acc, float4 *bb) {
  if (threadIdx.x == 0) {
    float lo[3], hi[3];
    for (int k = 0; k < 3; k++) {
      lo[k] = o2f(acc[k]);
      hi[k] = o2f(acc[3 + k]);
      if (!(lo[k] <= hi[k])) lo[k] = hi[k] = 0.f;
      lo[k] -= 1.f;
      hi[k] += 1.f;
    }
    bb[0] = make_float4(lo[0], lo[1], lo[2], 0.f);
    bb[1] = make_float4(hi[0], hi[1], hi[2], 0.f);
  }
}

// ---------------------------------------------------------------------------
// One-block LBVH build of a small per-frame tree (n <= kSmallBuildMax boxes or
// points): Morton codes, a bitonic sort of (code << 32 | index) keys in
// shared memory, the Karras hierarchy over the sorted keys, the primitives
// gathered in leaf order and the bottom-up boxes -- one launch where the
// device-wide path takes about twenty (code, four sort passes of three
// kernels, gather, hierarchy, flag reset, refit) whose launch latencies set
// the time of a small tree's update.  The index in the low key bits makes
// every key distinct, which is the tie-break of equal codes by position.
// Above 4096 primitives the one block's sort costs more than the launches
// it saves (measured: the city's 15k-primitive merged tree took 0.57 ms of
// update instead of 0.25 with the device-wide path), so larger trees take
// the cooperative build below (up to kCoopMax) or the device-wide path.
constexpr uint32_t kSmallBuildMax = 4096;
constexpr int kSmallBlock = 1024;

template <int KIND>
__global__ void __launch_bounds__(kSmallBlock) k_small_build(
    const float4 *a, const float4 *b, uint32_t n, uint32_t np2, const float4 *bb, float4 *prims,
    float4 *nodes, uint32_t *leaf_parent, float pad) {
  extern __shared__ unsigned long long sk[];   // np2 keys, then n arrival counters
  uint32_t *sflag = reinterpret_cast<uint32_t *>(sk + np2);
  const uint32_t tid = threadIdx.x;
  for (uint32_t i = tid; i < np2; i += blockDim.x) {
    unsigned long long key = ~0ull;
    if (i < n) {
      const float4 p = a[i];
      float3 c = f3(p);
      if (KIND == PRIM_BOX) {
        const float4 q = b[i];
        c = make_float3(0.5f * (p.x + q.x), 0.5f * (p.y + q.y), 0.5f * (p.z + q.z));
      }
      key = (unsigned long long)morton_code<kMortonBitsDyn>(c, bb) << 32 | i;
    }
    sk[i] = key;
  }
  for (uint32_t i = tid; i < n; i += blockDim.x) sflag[i] = 0u;
  __syncthreads();
  for (uint32_t k = 2; k <= np2; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = tid; i < (np2 >> 1); i += blockDim.x) {
        const uint32_t lo = 2u * i - (i & (j - 1u)), hi = lo + j;
        const unsigned long long x = sk[lo], y = sk[hi];
        if ((x > y) == ((lo & k) == 0u)) {
          sk[lo] = y;
          sk[hi] = x;
        }
      }
      __syncthreads();
    }
  }
  // primitives in leaf order (the source index kept in .w)
  for (uint32_t g = tid; g < n; g += blockDim.x) {
    const uint32_t src = (uint32_t)sk[g];
    const float4 p = a[src];
    if (KIND == PRIM_BOX) {
      const float4 q = b[src];
      prims[2ull * g + 0] = make_float4(p.x, p.y, p.z, __uint_as_float(src));
      prims[2ull * g + 1] = make_float4(q.x, q.y, q.z, 0.f);
    } else {
      prims[g] = make_float4(p.x, p.y, p.z, __uint_as_float(src));
    }
  }
  if (n < 2) return;
  // hierarchy: inner node i over the sorted keys (all distinct: the index
  // is in the low bits)
  const int nn = (int)n;
  for (int i = (int)tid; i < nn - 1; i += (int)blockDim.x)
    hierarchy_node([](int q) { return (uint64_t)sk[q]; }, nn, i, nodes, leaf_parent);
  __threadfence_block();
  __syncthreads();
  // bottom-up boxes: the second thread to reach a node merges its children
  for (uint32_t g = tid; g < n; g += blockDim.x) {
    Box bx = prim_box<KIND>(prims, g);
    bx.lo = make_float3(bx.lo.x - pad, bx.lo.y - pad, bx.lo.z - pad);
    bx.hi = make_float3(bx.hi.x + pad, bx.hi.y + pad, bx.hi.z + pad);
    int code = (int)__ldcg(leaf_parent + g);
    refit_up(bx, code, nodes, sflag);
  }
}

template <int KIND>
cudaError_t small_build(BVHBuf &b, const float4 *a, const float4 *bx, uint32_t n,
                        const float4 *bbox, cudaStream_t s) {
  uint32_t np2 = 2;
  while (np2 < n) np2 <<= 1;
  const size_t smem = sizeof(unsigned long long) * np2 + sizeof(uint32_t) * n;
  static_assert(sizeof(unsigned long long) * kSmallBuildMax + sizeof(uint32_t) * kSmallBuildMax <=
                    48 * 1024,
                "the one-block build fits the default shared-memory limit");
  emrt::note_launch(), k_small_build<KIND><<<1, kSmallBlock, smem, s>>>(a, bx, n, np2, bbox, b.prims,
                                                                       b.nodes, b.leaf_parent, b.pad);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-frame trees of kSmallBuildMax + 1 .. kCoopMax primitives: the steps of
// the device-wide build (Morton codes, four stable 8-bit radix passes over
// the 30-bit codes, gather, hierarchy, bottom-up boxes) in one cooperative
// launch, separated by a grid barrier, instead of ~18 launches and memsets
// whose latencies set a 5-15k primitive tree's build time.  Each block owns
// one tile of at most kCoopTile keys; a radix pass counts the tile's digits,
// and after the barrier every block sums the counts of all blocks (its own
// offsets: the digits' totals and the counts of the blocks before it) and
// scatters its tile, ranking equal digits by tile position, so every pass is
// stable and the sorted order, the tree and every query result are those of
// the device-wide path.  The barrier's wait is bounded: past kBarrierSpins
// polls the block records ERR_WAIT and the build stops (the cooperative
// launch keeps all blocks resident, so the bound is only a safety net).
constexpr uint32_t kCoopMax = 65536;
constexpr int kCoopBlock = 256;
constexpr uint32_t kCoopTile = 512;
constexpr uint32_t kBarrierSpins = 1u << 19;  // polls of ~1.4 us: about 0.7 s

// bar[0]: arrivals, bar[1]: generation, bar[2]: gave-up flag (zeroed
// before the launch)
__device__ inline bool grid_barrier(uint32_t *bar, uint32_t nb, uint32_t *err_word) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t *gen = bar + 1;
    const uint32_t g = *gen;
    __threadfence();
    bool ok = true;
    if (atomicAdd(bar, 1u) == nb - 1u) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      uint32_t it = 0;
      while (*gen == g) {
        if (++it > kBarrierSpins || *(volatile uint32_t *)(bar + 2)) {
          ok = false;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    if (!ok) {
      atomicExch(bar + 2, 1u);
      if (err_word) atomicOr(err_word, ERR_WAIT);
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <int KIND>
__device__ inline float3 dyn_centre(const float4 *a, const float4 *b, uint32_t i) {
  const float4 p = a[i];
  if (KIND == PRIM_BOX) {
    const float4 q = b[i];
    return make_float3(0.5f * (p.x + q.x), 0.5f * (p.y + q.y), 0.5f * (p.z + q.z));
  }
  return f3(p);
}

template <int KIND>
__global__ void __launch_bounds__(kCoopBlock) k_coop_build(
    const float4 *a, const float4 *bx, uint32_t n, const float4 *bb, KeyW<2> *k0, uint32_t *i0,
    KeyW<2> *k1, uint32_t *i1, uint32_t *hist, float4 *prims, float4 *nodes,
    uint32_t *leaf_parent, uint32_t *flags, float pad, uint32_t *bar, uint32_t *err_word) {
  __shared__ uint32_t s_code[kCoopTile], s_idx[kCoopTile];
  __shared__ uint32_t s_base[256], s_pre[256];
  const uint32_t nb = gridDim.x, blk = blockIdx.x, tid = threadIdx.x;
  const uint32_t tile = (n + nb - 1) / nb;  // <= kCoopTile (host check)
  const uint32_t t0 = min(blk * tile, n), tn = min(t0 + tile, n) - t0;
  for (uint32_t t = tid; t < tn; t += blockDim.x) {
    s_code[t] = (uint32_t)morton_code<kMortonBitsDyn>(dyn_centre<KIND>(a, bx, t0 + t), bb);
    s_idx[t] = t0 + t;
  }
  // LSD radix sort, 8 bits a pass; passes write k1/i1, k0/i0, k1/i1, k0/i0
  for (int pass = 0; pass < 4; pass++) {
    const int shift = 8 * pass;
    KeyW<2> *ko = (pass & 1) ? k0 : k1;
    uint32_t *io = (pass & 1) ? i0 : i1;
    for (uint32_t d = tid; d < 256; d += blockDim.x) s_base[d] = 0u;
    __syncthreads();
    for (uint32_t t = tid; t < tn; t += blockDim.x) atomicAdd(&s_base[(s_code[t] >> shift) & 255u], 1u);
    __syncthreads();
    for (uint32_t d = tid; d < 256; d += blockDim.x) hist[256ull * blk + d] = s_base[d];
    if (!grid_barrier(bar, nb, err_word)) return;
    for (uint32_t d = tid; d < 256; d += blockDim.x) {
      uint32_t tot = 0, pre = 0;
      for (uint32_t j = 0; j < nb; j++) {
        const uint32_t v = __ldcg(hist + 256ull * j + d);
        tot += v;
        pre += j < blk ? v : 0u;
      }
      s_base[d] = tot;
      s_pre[d] = pre;
    }
    __syncthreads();
    if (tid == 0) {  // exclusive scan of the digit totals
      uint32_t run = 0;
      for (uint32_t d = 0; d < 256; d++) {
        const uint32_t v = s_base[d];
        s_base[d] = run;
        run += v;
      }
    }
    __syncthreads();
    for (uint32_t t = tid; t < tn; t += blockDim.x) {
      const uint32_t dg = (s_code[t] >> shift) & 255u;
      uint32_t r = 0;
      for (uint32_t u = 0; u < t; u++) r += ((s_code[u] >> shift) & 255u) == dg;
      const uint32_t dst = s_base[dg] + s_pre[dg] + r;
      KeyW<2> kk;
      kk.w[0] = s_code[t];
      kk.w[1] = 0u;
      ko[dst] = kk;
      io[dst] = s_idx[t];
    }
    if (!grid_barrier(bar, nb, err_word)) return;
    if (pass < 3) {
      for (uint32_t t = tid; t < tn; t += blockDim.x) {
        s_code[t] = __ldcg(&ko[t0 + t].w[0]);
        s_idx[t] = __ldcg(io + t0 + t);
      }
      __syncthreads();
    }
  }
  // primitives in leaf order, arrival counters cleared, hierarchy
  const uint32_t stride = nb * blockDim.x;
  for (uint32_t g = blk * blockDim.x + tid; g < n; g += stride) {
    const uint32_t src = __ldcg(i0 + g);
    const float4 p = a[src];
    if (KIND == PRIM_BOX) {
      const float4 q = bx[src];
      prims[2ull * g + 0] = make_float4(p.x, p.y, p.z, __uint_as_float(src));
      prims[2ull * g + 1] = make_float4(q.x, q.y, q.z, 0.f);
    } else {
      prims[g] = make_float4(p.x, p.y, p.z, __uint_as_float(src));
    }
    flags[g] = 0u;
  }
  for (uint32_t i = blk * blockDim.x + tid; i + 1 < n; i += stride)
    hierarchy_node([k0](int q) { return (uint64_t)__ldcg(&k0[q].w[0]); }, (int)n, (int)i, nodes,
                   leaf_parent);
  if (!grid_barrier(bar, nb, err_word)) return;
  // bottom-up boxes (this thread gathered primitive g itself)
  for (uint32_t g = blk * blockDim.x + tid; g < n; g += stride) {
    Box b = prim_box<KIND>(prims, g);
    b.lo = make_float3(b.lo.x - pad, b.lo.y - pad, b.lo.z - pad);
    b.hi = make_float3(b.hi.x + pad, b.hi.y + pad, b.hi.z + pad);
    refit_up(b, (int)__ldcg(leaf_parent + g), nodes, flags);
  }
}

int g_sms = 0;
int sm_count() {
  if (!g_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 1;
  }
  return g_sms;
}

// blocks of the cooperative build of n primitives (tiles of about 128 keys,
// at most one block per SM, at least ceil(n / kCoopTile))
uint32_t coop_grid(uint32_t n) {
  const uint32_t g = std::min<uint32_t>((uint32_t)sm_count(), ceil_div(n, 128u));
  return std::max<uint32_t>(g, ceil_div(n, kCoopTile));
}

template <int KIND>
cudaError_t coop_build(BVHBuf &b, const float4 *a, const float4 *bx, uint32_t n,
                       const float4 *bbox, cudaStream_t s) {
  uint32_t grid = coop_grid(n);
  cudaMemsetAsync(b.coop_bar, 0, 3 * sizeof(uint32_t), s);
  void *args[] = {(void *)&a,        (void *)&bx,          (void *)&n,       (void *)&bbox,
                  (void *)&b.keys,   (void *)&b.idx,       (void *)&b.keys2, (void *)&b.idx2,
                  (void *)&b.coop_hist, (void *)&b.prims,  (void *)&b.nodes, (void *)&b.leaf_parent,
                  (void *)&b.flags,  (void *)&b.pad,       (void *)&b.coop_bar, (void *)&b.err_word};
  emrt::note_launch();
  return cudaLaunchCooperativeKernel((const void *)k_coop_build<KIND>, dim3(grid),
                                     dim3(kCoopBlock), args, 0, s);
}

// grid_barrier with nb arrivals expected from a launch of `blocks` blocks:
// with nb > blocks the barrier cannot complete and every block gives up
__global__ void k_barrier_selftest(uint32_t *bar, uint32_t nb, uint32_t *err_word,
                                   uint32_t *passed) {
  if (grid_barrier(bar, nb, err_word) && threadIdx.x == 0) atomicAdd(passed, 1u);
}

template <int KIND>
cudaError_t finish_build(BVHBuf &b, cudaStream_t s) {
  uint32_t n = b.n;
  if (n >= 2) {
    emrt::note_launch(), k_hierarchy<<<ceil_div(n - 1, 256), 256, 0, s>>>(b.keys, (int)n, b.nodes, b.leaf_parent);
    cudaMemsetAsync(b.flags, 0, sizeof(uint32_t) * n, s);
    emrt::note_launch(), k_refit<KIND><<<ceil_div(n, 256), 256, 0, s>>>(b.prims, n, b.nodes, b.leaf_parent, b.flags, b.pad);
  }
  return cudaGetLastError();
}

__global__ void k_set_u32(uint32_t *p, uint32_t v) { *p = v; }

template <int KIND>
cudaError_t sort_codes(BVHBuf &b, uint32_t *hist, cudaStream_t s) {
  emrt::note_launch(), k_set_u32<<<1, 1, 0, s>>>(b.d_n, b.n);
  const int bits = 3 * (KIND == PRIM_TRI ? kMortonBitsTri : kMortonBitsDyn);
  bool alt = radix_sort<2>(b.d_n, b.keys, b.idx, b.keys2, b.idx2, bits, hist, s, b.n);
  if (alt) {
    std::swap(b.keys, b.keys2);
    std::swap(b.idx, b.idx2);
  }
  return cudaGetLastError();
}

}  // namespace

BVHView BVHBuf::view() const {
  BVHView v;
  v.nodes8 = nodes8;
  v.prims8 = prims8;
  v.nodes = nodes;
  v.prims = prims;
  v.root = n >= 2 ? 0 : ~0;
  v.n_prims = n;
  v.leaf_bits = leaf_bits;
  return v;
}

cudaError_t bvh_alloc(BVHBuf &b, PrimKind kind, uint32_t cap) {
  bvh_free(b);
  b.kind = kind;
  b.cap = cap < 2 ? 2 : cap;
  int words = kind == PRIM_TRI ? 3 : (kind == PRIM_BOX ? 2 : 1);
  cudaError_t e = cudaSuccess;
  auto A = [&](void **p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
  A((void **)&b.nodes, sizeof(float4) * 4 * (size_t)b.cap);
  A((void **)&b.prims, sizeof(float4) * words * (size_t)b.cap);
  A((void **)&b.leaf_parent, sizeof(uint32_t) * b.cap);
  A((void **)&b.flags, sizeof(uint32_t) * b.cap);
  A((void **)&b.keys, sizeof(KeyW<2>) * b.cap);
  A((void **)&b.keys2, sizeof(KeyW<2>) * b.cap);
  A((void **)&b.idx, sizeof(uint32_t) * b.cap);
  A((void **)&b.idx2, sizeof(uint32_t) * b.cap);
  A((void **)&b.d_n, sizeof(uint32_t));
  if (kind != PRIM_TRI && b.cap > kSmallBuildMax) {
    A((void **)&b.coop_hist, sizeof(uint32_t) * 256 * (size_t)coop_grid(std::min(b.cap, kCoopMax)));
    A((void **)&b.coop_bar, sizeof(uint32_t) * 4);
  }
  return e;
}

void bvh_free(BVHBuf &b) {
  cudaFree(b.nodes); cudaFree(b.prims); cudaFree(b.leaf_parent); cudaFree(b.flags);
  cudaFree(b.keys); cudaFree(b.keys2); cudaFree(b.idx); cudaFree(b.idx2); cudaFree(b.d_n);
  cudaFree(b.coop_hist); cudaFree(b.coop_bar);
  b.coop_hist = b.coop_bar = nullptr;
  cudaFree(b.nodes8);
  cudaFree(b.prims8);
  b.nodes8 = nullptr;
  b.prims8 = nullptr;
  b.n8 = 0;
  b.nodes = b.prims = nullptr;
  b.leaf_parent = b.flags = b.idx = b.idx2 = b.d_n = nullptr;
  b.keys = b.keys2 = nullptr;
  b.n = b.cap = 0;
}

cudaError_t bvh_build_tris(BVHBuf &b, const float *tri_xyz, const uint32_t *tri_face, uint32_t n,
                           const float4 *bbox, uint32_t *hist, cudaStream_t s) {
  b.n = n;
  if (n == 0) return cudaSuccess;
  emrt::note_launch(), k_morton_tris<<<ceil_div(n, 256), 256, 0, s>>>(tri_xyz, n, bbox, b.keys, b.idx);
  sort_codes<PRIM_TRI>(b, hist, s);
  emrt::note_launch(), k_gather_tris<<<ceil_div(n, 256), 256, 0, s>>>(tri_xyz, tri_face, b.idx, n, b.prims);
  return finish_build<PRIM_TRI>(b, s);
}

cudaError_t grid_barrier_selftest(uint32_t missing, uint32_t *passed, uint32_t *timed_out) {
  const uint32_t blocks = 4;
  uint32_t *d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(uint32_t) * 6);  // bar[4], err word, passed
  if (e != cudaSuccess) return e;
  cudaMemset(d, 0, sizeof(uint32_t) * 6);
  uint32_t *bar = d, *err = d + 4, *pass = d + 5;
  uint32_t nb = blocks + missing;
  void *args[] = {(void *)&bar, (void *)&nb, (void *)&err, (void *)&pass};
  emrt::note_launch();
  e = cudaLaunchCooperativeKernel((const void *)k_barrier_selftest, dim3(blocks), dim3(kCoopBlock),
                                  args, 0, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  uint32_t h[6] = {0, 0, 0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  *passed = h[5];
  *timed_out = (h[4] & ERR_WAIT) ? 1u : 0u;
  return e;
}

cudaError_t bvh_build_boxes(BVHBuf &b, const float4 *lo, const float4 *hi, uint32_t n,
                            const float4 *bbox, uint32_t *hist, cudaStream_t s) {
  b.n = n;
  if (n == 0) return cudaSuccess;
  if (n <= kSmallBuildMax) return small_build<PRIM_BOX>(b, lo, hi, n, bbox, s);
  if (n <= kCoopMax && b.coop_bar) return coop_build<PRIM_BOX>(b, lo, hi, n, bbox, s);
  emrt::note_launch(), k_morton_boxes<<<ceil_div(n, 256), 256, 0, s>>>(lo, hi, n, bbox, b.keys, b.idx);
  sort_codes<PRIM_BOX>(b, hist, s);
  emrt::note_launch(), k_gather_boxes<<<ceil_div(n, 256), 256, 0, s>>>(lo, hi, b.idx, n, b.prims);
  return finish_build<PRIM_BOX>(b, s);
}

cudaError_t bvh_refit_boxes(BVHBuf &b, const float4 *lo, const float4 *hi, cudaStream_t s) {
  uint32_t n = b.n;
  if (n == 0) return cudaSuccess;
  emrt::note_launch(), k_move_boxes<<<ceil_div(n, 256), 256, 0, s>>>(lo, hi, n, b.prims);
  if (n >= 2) {
    cudaMemsetAsync(b.flags, 0, sizeof(uint32_t) * n, s);
    emrt::note_launch(), k_refit<PRIM_BOX><<<ceil_div(n, 256), 256, 0, s>>>(b.prims, n, b.nodes, b.leaf_parent, b.flags, b.pad);
  }
  return cudaGetLastError();
}

cudaError_t bvh_build_points(BVHBuf &b, const float4 *pts, uint32_t n, const float4 *bbox,
                             uint32_t *hist, cudaStream_t s) {
  b.n = n;
  if (n == 0) return cudaSuccess;
  if (n <= kSmallBuildMax) return small_build<PRIM_POINT>(b, pts, nullptr, n, bbox, s);
  if (n <= kCoopMax && b.coop_bar) return coop_build<PRIM_POINT>(b, pts, nullptr, n, bbox, s);
  emrt::note_launch(), k_morton_points<<<ceil_div(n, 256), 256, 0, s>>>(pts, n, bbox, b.keys, b.idx);
  sort_codes<PRIM_POINT>(b, hist, s);
  emrt::note_launch(), k_gather_points<<<ceil_div(n, 256), 256, 0, s>>>(pts, b.idx, n, b.prims);
  return finish_build<PRIM_POINT>(b, s);
}

// ---------------------------------------------------------------------------
// Binned SAH top-down build (static triangles; built once).  Level by level,
// one block per node range: centroid bounds, 64 bins along each axis,
// surface-area-heuristic sweep over all three, stable partition of the range.  Ranges of one
// triangle become leaves.  Writes the same node format as the LBVH (child
// codes and parent links); boxes are filled by the bottom-up refit.
namespace {

constexpr int kSahBins = 64;
constexpr int kSahBlock = 256;
constexpr int kSahMaxDepth = 60;  // levels; the traversal stack holds 64 entries
// ranges of up to this many clusters become leaves (a cluster is one
// triangle or the two triangles of a quad face; on the city one cluster per
// leaf is fastest: leaves of up to 4 triangles chosen by the SAH cut node
// visits 29.0 -> 25.7 per segment but raised triangle tests 2.5 -> 6.7 and
// the traversal 16.0 -> 18.8 ms)
constexpr uint32_t kSahLeafMax = 1;

struct SahTask {
  uint32_t b, e, node, pad;
};

__global__ void k_tri_bounds(const float *t, uint32_t n, float4 *cen, float4 *lo, float4 *hi,
                             uint32_t *perm) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float *v = t + 9ull * i;
  float3 a = make_float3(fminf(v[0], fminf(v[3], v[6])), fminf(v[1], fminf(v[4], v[7])),
                         fminf(v[2], fminf(v[5], v[8])));
  float3 b = make_float3(fmaxf(v[0], fmaxf(v[3], v[6])), fmaxf(v[1], fmaxf(v[4], v[7])),
                         fmaxf(v[2], fmaxf(v[5], v[8])));
  lo[i] = make_float4(a.x, a.y, a.z, 0.f);
  hi[i] = make_float4(b.x, b.y, b.z, 0.f);
  cen[i] = make_float4((v[0] + v[3] + v[6]) * (1.f / 3.f), (v[1] + v[4] + v[7]) * (1.f / 3.f),
                       (v[2] + v[5] + v[8]) * (1.f / 3.f), 0.f);
  perm[i] = i;
}

// Leaf clusters of the SAH build: two consecutive triangles of one face with
// the same bounding box (the two halves of a planar quad -- a wall, a ground
// tile) form one leaf, every other triangle a leaf of its own.  The pair's
// two tests are those the two single-triangle leaves would get whenever
// their common box is entered; the inner node that split them is saved.
// Triangle i+1 joins i when the pair matches and i does not itself join
// i-1, so pairs never overlap.
__device__ inline bool same_box_pair(const float *t, const uint32_t *tri_face, uint32_t n,
                                     uint32_t i) {
  if (i + 1 >= n || tri_face[i] != tri_face[i + 1]) return false;
  const float *a = t + 9ull * i, *b = a + 9;
  for (int d = 0; d < 3; d++) {
    const float alo = fminf(a[d], fminf(a[3 + d], a[6 + d]));
    const float ahi = fmaxf(a[d], fmaxf(a[3 + d], a[6 + d]));
    const float blo = fminf(b[d], fminf(b[3 + d], b[6 + d]));
    const float bhi = fmaxf(b[d], fmaxf(b[3 + d], b[6 + d]));
    if (alo != blo || ahi != bhi) return false;
  }
  return true;
}

__device__ inline bool joins_previous(const float *t, const uint32_t *tri_face, uint32_t n,
                                      uint32_t i) {
  return i > 0 && same_box_pair(t, tri_face, n, i - 1) &&
         !(i > 1 && same_box_pair(t, tri_face, n, i - 2));
}

// flag[i] = 1 when triangle i starts a cluster (pairing on or off)
__global__ void k_cluster_flags(const float *t, const uint32_t *tri_face, uint32_t n, int pairs,
                                uint32_t *flag) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  flag[i] = (!pairs || !joins_previous(t, tri_face, n, i)) ? 1u : 0u;
}

// cluster list (first triangle, second triangle or ~0) and the SAH inputs:
// box of the cluster, centroid = mean of its triangles' centroids
__global__ void k_cluster_bounds(const float *t, const uint32_t *tri_face, uint32_t n, int pairs,
                                 const uint32_t *flag, const uint32_t *pos, uint2 *cl, float4 *cen,
                                 float4 *lo, float4 *hi, uint32_t *perm) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !flag[i]) return;
  const uint32_t j = (pairs && joins_previous(t, tri_face, n, i + 1)) ? i + 1 : 0xffffffffu;
  const uint32_t c = pos[i];
  cl[c] = make_uint2(i, j);
  float a[3] = {3.4e38f, 3.4e38f, 3.4e38f}, b[3] = {-3.4e38f, -3.4e38f, -3.4e38f}, m[3] = {0, 0, 0};
  const uint32_t tt[2] = {i, j};
  const int k = j == 0xffffffffu ? 1 : 2;
  for (int q = 0; q < k; q++) {
    const float *v = t + 9ull * tt[q];
    for (int d = 0; d < 3; d++) {
      a[d] = fminf(a[d], fminf(v[d], fminf(v[3 + d], v[6 + d])));
      b[d] = fmaxf(b[d], fmaxf(v[d], fmaxf(v[3 + d], v[6 + d])));
      m[d] += (v[d] + v[3 + d] + v[6 + d]) * (1.f / 3.f);
    }
  }
  const float w = 1.f / (float)k;
  lo[c] = make_float4(a[0], a[1], a[2], 0.f);
  hi[c] = make_float4(b[0], b[1], b[2], 0.f);
  cen[c] = make_float4(m[0] * w, m[1] * w, m[2] * w, 0.f);
  perm[c] = c;
}

__global__ void k_cluster_sizes(const uint2 *cl, const uint32_t *perm, uint32_t nc, uint32_t *sz) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nc) sz[p] = cl[perm[p]].y == 0xffffffffu ? 1u : 2u;
}

// triangle order of the leaves, triangle leaf parents and the final leaf
// codes ~(first triangle << 2 | count - 1)
__global__ void k_cluster_expand(const uint2 *cl, const uint32_t *perm, const uint32_t *tstart,
                                 const uint32_t *lp_cl, uint32_t nc, uint32_t *tri_idx,
                                 uint32_t *leaf_parent, float4 *nodes) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nc) return;
  const uint2 c = cl[perm[p]];
  const uint32_t t0 = tstart[p], lp = lp_cl[p];
  const uint32_t k = c.y == 0xffffffffu ? 1u : 2u;
  tri_idx[t0] = c.x;
  leaf_parent[t0] = lp;
  if (k == 2u) {
    tri_idx[t0 + 1] = c.y;
    leaf_parent[t0 + 1] = 0xffffffffu;
  }
  reinterpret_cast<int *>(nodes + 4ll * (lp >> 1) + 3)[lp & 1u] = ~(int)(t0 << 2 | (k - 1u));
}

__device__ inline float sel(float4 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

__device__ inline void block_minmax(float &mn, float &mx, float *sh) {
  for (int o = 16; o; o >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) { sh[w] = mn; sh[32 + w] = mx; }
  __syncthreads();
  if (threadIdx.x < 32) {
    int nw = blockDim.x >> 5;
    mn = threadIdx.x < nw ? sh[threadIdx.x] : 3.4e38f;
    mx = threadIdx.x < nw ? sh[32 + threadIdx.x] : -3.4e38f;
    for (int o = 16; o; o >>= 1) {
      mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (threadIdx.x == 0) { sh[0] = mn; sh[32] = mx; }
  }
  __syncthreads();
  mn = sh[0];
  mx = sh[32];
  __syncthreads();
}

__device__ inline uint32_t f2o_d(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ inline float o2f_d(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void __launch_bounds__(kSahBlock) k_sah_level(
    const SahTask *tasks, const uint32_t *n_tasks, const float4 *cen, const float4 *blo,
    const float4 *bhi, uint32_t *perm, uint32_t *tmp, float4 *nodes, uint32_t *leaf_parent,
    SahTask *out, uint32_t *n_out, uint32_t *n_alloc) {
  __shared__ float sh[64];
  __shared__ uint32_t bcnt[3][kSahBins];
  __shared__ uint32_t blo_s[3][kSahBins][3], bhi_s[3][kSahBins][3];
  __shared__ int s_axis, s_split;
  __shared__ float s_lo, s_ext;
  __shared__ uint32_t s_carry, s_wsum[kSahBlock / 32];
  if (blockIdx.x >= *n_tasks) return;
  SahTask T = tasks[blockIdx.x];
  const uint32_t b = T.b, e = T.e, cnt = e - b;
  // centroid bounds
  float lo3[3], hi3[3];
  for (int k = 0; k < 3; k++) {
    float mn = 3.4e38f, mx = -3.4e38f;
    for (uint32_t i = b + threadIdx.x; i < e; i += blockDim.x) {
      float c = sel(cen[perm[i]], k);
      mn = fminf(mn, c);
      mx = fmaxf(mx, c);
    }
    block_minmax(mn, mx, sh);
    lo3[k] = mn;
    hi3[k] = mx;
  }
  // bins along every axis of non-zero centroid extent; the split with the
  // lowest surface-area cost over all three axes is taken
  for (int t = threadIdx.x; t < 3 * kSahBins; t += blockDim.x) {
    const int k = t / kSahBins, q = t % kSahBins;
    bcnt[k][q] = 0;
    for (int c = 0; c < 3; c++) {
      blo_s[k][q][c] = 0xffffffffu;
      bhi_s[k][q][c] = 0u;
    }
  }
  if (threadIdx.x == 0) s_split = -1;
  __syncthreads();
  float ext3[3];
  for (int k = 0; k < 3; k++) ext3[k] = hi3[k] - lo3[k];
  for (uint32_t i = b + threadIdx.x; i < e; i += blockDim.x) {
    const uint32_t p = perm[i];
    const float4 c4 = cen[p], a = blo[p], z = bhi[p];
    for (int k = 0; k < 3; k++) {
      if (!(ext3[k] > 0.f)) continue;
      const int bin = min(kSahBins - 1, (int)((sel(c4, k) - lo3[k]) / ext3[k] * kSahBins));
      atomicAdd(&bcnt[k][bin], 1u);
      for (int c = 0; c < 3; c++) {
        atomicMin(&blo_s[k][bin][c], f2o_d(sel(a, c)));
        atomicMax(&bhi_s[k][bin][c], f2o_d(sel(z, c)));
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // SAH sweep over the 31 bin boundaries of each axis
    float best = 3.4e38f;
    int bax = -1, bs = -1;
    for (int k = 0; k < 3; k++) {
      if (!(ext3[k] > 0.f)) continue;
      float rl[kSahBins][3], rh[kSahBins][3];
      uint32_t rc[kSahBins];
      float l3[3] = {3.4e38f, 3.4e38f, 3.4e38f}, h3[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
      uint32_t c = 0;
      for (int q = kSahBins - 1; q >= 0; q--) {
        if (bcnt[k][q]) {
          for (int d = 0; d < 3; d++) {
            l3[d] = fminf(l3[d], o2f_d(blo_s[k][q][d]));
            h3[d] = fmaxf(h3[d], o2f_d(bhi_s[k][q][d]));
          }
        }
        c += bcnt[k][q];
        rc[q] = c;
        for (int d = 0; d < 3; d++) { rl[q][d] = l3[d]; rh[q][d] = h3[d]; }
      }
      float a3[3] = {3.4e38f, 3.4e38f, 3.4e38f}, z3[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
      uint32_t lc = 0;
      for (int q = 0; q < kSahBins - 1; q++) {
        if (bcnt[k][q]) {
          for (int d = 0; d < 3; d++) {
            a3[d] = fminf(a3[d], o2f_d(blo_s[k][q][d]));
            z3[d] = fmaxf(z3[d], o2f_d(bhi_s[k][q][d]));
          }
        }
        lc += bcnt[k][q];
        const uint32_t rcnt = rc[q + 1];
        if (lc == 0 || rcnt == 0) continue;
        const float dl[3] = {z3[0] - a3[0], z3[1] - a3[1], z3[2] - a3[2]};
        const float dr[3] = {rh[q + 1][0] - rl[q + 1][0], rh[q + 1][1] - rl[q + 1][1],
                             rh[q + 1][2] - rl[q + 1][2]};
        const float al = dl[0] * dl[1] + dl[1] * dl[2] + dl[2] * dl[0];
        const float ar = dr[0] * dr[1] + dr[1] * dr[2] + dr[2] * dr[0];
        const float cost = al * lc + ar * rcnt;
        if (cost < best) { best = cost; bax = k; bs = q + 1; }
      }
    }
    s_split = bs;
    s_axis = bax < 0 ? 0 : bax;
    s_lo = lo3[s_axis];
    s_ext = ext3[s_axis];
  }
  __syncthreads();
  const int ax = s_axis;
  const float lo = s_lo, ext = s_ext;
  const int split = s_split;
  // stable partition of the range into tmp, then back into perm
  uint32_t nl;
  if (split < 0) {
    nl = cnt / 2;  // degenerate: all centroids in one bin; any split is valid
  } else {
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint32_t r0 = b; r0 < e; r0 += blockDim.x) {
      uint32_t i = r0 + threadIdx.x;
      uint32_t p = 0;
      bool left = false;
      if (i < e) {
        p = perm[i];
        left = min(kSahBins - 1, (int)((sel(cen[p], ax) - lo) / ext * kSahBins)) < split;
      }
      uint32_t m = __ballot_sync(0xffffffffu, left);
      int w = threadIdx.x >> 5, l = threadIdx.x & 31;
      if (l == 0) s_wsum[w] = __popc(m);
      __syncthreads();
      uint32_t before = s_carry;
      for (int q = 0; q < w; q++) before += s_wsum[q];
      before += __popc(m & ((1u << l) - 1u));
      if (i < e && left) tmp[b + before] = p;
      __syncthreads();
      if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) s_carry += s_wsum[q];
      __syncthreads();
    }
    nl = s_carry;
    __syncthreads();  // every thread has read the left count before the reset
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint32_t r0 = b; r0 < e; r0 += blockDim.x) {
      uint32_t i = r0 + threadIdx.x;
      uint32_t p = 0;
      bool right = false;
      if (i < e) {
        p = perm[i];
        right = min(kSahBins - 1, (int)((sel(cen[p], ax) - lo) / ext * kSahBins)) >= split;
      }
      uint32_t m = __ballot_sync(0xffffffffu, right);
      int w = threadIdx.x >> 5, l = threadIdx.x & 31;
      if (l == 0) s_wsum[w] = __popc(m);
      __syncthreads();
      uint32_t before = s_carry;
      for (int q = 0; q < w; q++) before += s_wsum[q];
      before += __popc(m & ((1u << l) - 1u));
      if (i < e && right) tmp[b + nl + before] = p;
      __syncthreads();
      if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) s_carry += s_wsum[q];
      __syncthreads();
    }
    for (uint32_t i = b + threadIdx.x; i < e; i += blockDim.x) perm[i] = tmp[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t rb[2] = {b, b + nl}, re[2] = {b + nl, e};
    int code[2];
    for (int side = 0; side < 2; side++) {
      const uint32_t rn = re[side] - rb[side];
      if (rn <= kSahLeafMax) {
        code[side] = ~(int)(rb[side] << 2 | (rn - 1));
        leaf_parent[rb[side]] = 2 * T.node + side;
        for (uint32_t q = 1; q < rn; q++) leaf_parent[rb[side] + q] = 0xffffffffu;
      } else {
        uint32_t ni = atomicAdd(n_alloc, 1u);
        code[side] = (int)ni;
        reinterpret_cast<int *>(nodes + 4ll * ni + 3)[2] = (int)(2 * T.node + side);
        uint32_t slot = atomicAdd(n_out, 1u);
        out[slot] = SahTask{rb[side], re[side], ni, 0u};
      }
    }
    int *n3 = reinterpret_cast<int *>(nodes + 4ll * T.node + 3);
    n3[0] = code[0];
    n3[1] = code[1];
    n3[3] = 0;
    if (T.node == 0) n3[2] = -1;
  }
}

}  // namespace

cudaError_t bvh_build_tris_sah(BVHBuf &b, const float *tri_xyz, const uint32_t *tri_face, uint32_t n,
                               cudaStream_t s) {
  b.n = n;
  if (n == 0) return cudaSuccess;
  cudaError_t e;
  float4 *cen = nullptr, *lo = nullptr, *hi = nullptr;
  uint32_t *tmp = nullptr, *ctr = nullptr, *cbuf = nullptr;
  uint2 *cl = nullptr;
  SahTask *tasks[2] = {nullptr, nullptr};
  if ((e = cudaMalloc(&cen, sizeof(float4) * n))) return e;
  if ((e = cudaMalloc(&lo, sizeof(float4) * n))) return e;
  if ((e = cudaMalloc(&hi, sizeof(float4) * n))) return e;
  if ((e = cudaMalloc(&tmp, sizeof(uint32_t) * n))) return e;
  if ((e = cudaMalloc(&tasks[0], sizeof(SahTask) * (n / 2 + 2)))) return e;
  if ((e = cudaMalloc(&tasks[1], sizeof(SahTask) * (n / 2 + 2)))) return e;
  if ((e = cudaMalloc(&ctr, sizeof(uint32_t) * 8))) return e;
  // flags, positions, cluster leaf parents, sizes, starts, scan partials
  if ((e = cudaMalloc(&cbuf, sizeof(uint32_t) * (5 * (size_t)n + kPrimGrid + 1)))) return e;
  if ((e = cudaMalloc(&cl, sizeof(uint2) * n))) return e;
  uint32_t *flag = cbuf, *pos = cbuf + n, *lp_cl = cbuf + 2 * (size_t)n, *sz = cbuf + 3 * (size_t)n,
           *tstart = cbuf + 4 * (size_t)n, *partial = cbuf + 5 * (size_t)n;
  // clusters: pairs kept together unless that leaves fewer than two leaves
  uint32_t nc = 0;
  for (int pairs = 1; pairs >= 0; pairs--) {
    emrt::note_launch(), k_cluster_flags<<<ceil_div(n, 256), 256, 0, s>>>(tri_xyz, tri_face, n, pairs, flag);
    emrt::note_launch(), k_set_u32<<<1, 1, 0, s>>>(ctr + 4, n);
    exclusive_scan(ctr + 4, flag, pos, ctr + 5, partial, s);
    cudaMemcpyAsync(&nc, ctr + 5, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) break;
    emrt::note_launch(), k_cluster_bounds<<<ceil_div(n, 256), 256, 0, s>>>(
        tri_xyz, tri_face, n, pairs, flag, pos, cl, cen, lo, hi, b.idx);
    if (nc >= 2 || n < 2) break;
  }
  if (!e && nc >= 2) {
    SahTask root{0u, nc, 0u, 0u};
    uint32_t init[4] = {1, 0, 1, 0};  // level sizes [0],[1]; nodes allocated [2]
    cudaMemcpyAsync(tasks[0], &root, sizeof(root), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(ctr, init, sizeof(init), cudaMemcpyHostToDevice, s);
    uint32_t n_level = 1, zero = 0;
    int cur = 0, levels = 0;
    for (; n_level && levels < kSahMaxDepth; levels++) {
      cudaMemcpyAsync(ctr + (cur ^ 1), &zero, sizeof(uint32_t), cudaMemcpyHostToDevice, s);
      emrt::note_launch(), k_sah_level<<<n_level, kSahBlock, 0, s>>>(
          tasks[cur], ctr + cur, cen, lo, hi, b.idx, tmp, b.nodes, lp_cl, tasks[cur ^ 1],
          ctr + (cur ^ 1), ctr + 2);
      cudaMemcpyAsync(&n_level, ctr + (cur ^ 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
      if ((e = cudaStreamSynchronize(s))) break;
      cur ^= 1;
    }
    // a tree deeper than the traversal stack can serve is not used: the
    // caller falls back to the LBVH
    if (!e && n_level) e = cudaErrorNotSupported;
    if (!e) {  // leaves of clusters -> leaves of triangles
      emrt::note_launch(), k_set_u32<<<1, 1, 0, s>>>(ctr + 4, nc);
      emrt::note_launch(), k_cluster_sizes<<<ceil_div(nc, 256), 256, 0, s>>>(cl, b.idx, nc, sz);
      exclusive_scan(ctr + 4, sz, tstart, ctr + 5, partial, s);
      emrt::note_launch(), k_cluster_expand<<<ceil_div(nc, 256), 256, 0, s>>>(
          cl, b.idx, tstart, lp_cl, nc, b.idx2, b.leaf_parent, b.nodes);
    }
  } else if (!e) {  // a single triangle
    emrt::note_launch(), k_set_u32<<<1, 1, 0, s>>>(b.idx2, 0u);
  }
  if (!e) {
    emrt::note_launch(), k_gather_tris<<<ceil_div(n, 256), 256, 0, s>>>(tri_xyz, tri_face, b.idx2, n, b.prims);
    if (n >= 2) {
      cudaMemsetAsync(b.flags, 0, sizeof(uint32_t) * n, s);
      emrt::note_launch(), k_refit<PRIM_TRI, true><<<ceil_div(n, 256), 256, 0, s>>>(b.prims, n, b.nodes, b.leaf_parent, b.flags, b.pad);
    }
    e = cudaStreamSynchronize(s);
    if (!e) b.leaf_bits = 2;
  }
  cudaFree(cen); cudaFree(lo); cudaFree(hi); cudaFree(tmp);
  cudaFree(tasks[0]); cudaFree(tasks[1]); cudaFree(ctr); cudaFree(cbuf);
  cudaFree(cl);
  if (e) return e;
  return cudaGetLastError();
}

cudaError_t bvh8_build(BVHBuf &b, cudaStream_t s) {
  cudaFree(b.nodes8);
  cudaFree(b.prims8);
  b.nodes8 = nullptr;
  b.prims8 = nullptr;
  b.n8 = 0;
  if (b.n < 2 || b.kind != PRIM_TRI) return cudaSuccess;
  cudaError_t e;
  if ((e = cudaMalloc(&b.nodes8, sizeof(uint4) * 5 * (size_t)(b.n - 1)))) return e;
  if ((e = cudaMalloc(&b.prims8, sizeof(float4) * 3 * (size_t)b.n))) return e;
  uint32_t *buf = nullptr;  // two level lists (binary index, wide index) + counters
  if ((e = cudaMalloc(&buf, sizeof(uint32_t) * (4 * (size_t)b.n + 4)))) return e;
  uint32_t *lb[2] = {buf, buf + b.n}, *ld[2] = {buf + 2 * b.n, buf + 3 * b.n};
  uint32_t *ctr = buf + 4 * b.n;  // [0],[1]: level sizes, [2]: nodes, [3]: triangles
  uint32_t init[4] = {1, 0, 1, 0};
  uint32_t zero = 0;
  cudaMemcpyAsync(ctr, init, sizeof(init), cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(lb[0], 0, sizeof(uint32_t), s);
  cudaMemsetAsync(ld[0], 0, sizeof(uint32_t), s);
  uint32_t n_level = 1;
  int cur = 0;
  for (int guard = 0; n_level && guard < 4096; guard++) {
    cudaMemcpyAsync(ctr + (cur ^ 1), &zero, sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    emrt::note_launch(), k_wide8<<<ceil_div(n_level, 64), 64, 0, s>>>(
        b.nodes, b.prims, b.leaf_bits, lb[cur], ld[cur], ctr + cur, b.nodes8, b.prims8,
        lb[cur ^ 1], ld[cur ^ 1], ctr + (cur ^ 1), ctr + 2, ctr + 3);
    cudaMemcpyAsync(&n_level, ctr + (cur ^ 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) break;
    cur ^= 1;
  }
  cudaMemcpyAsync(&b.n8, ctr + 2, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  cudaFree(buf);
  if (e) return e;
  if (b.n8 >= (1u << 24)) {  // child indices hold 24 bits: no wide tree
    cudaFree(b.nodes8);
    cudaFree(b.prims8);
    b.nodes8 = nullptr;
    b.prims8 = nullptr;
    b.n8 = 0;
  }
  return cudaGetLastError();
}

void bbox_of_tris(const float *tri_xyz, uint32_t n, float4 *bbox, cudaStream_t s) {
  uint32_t *acc = reinterpret_cast<uint32_t *>(bbox + 2);  // 6 words of scratch after bbox
  emrt::note_launch(), k_bbox_init<<<1, 32, 0, s>>>(acc);
  if (n) emrt::note_launch(), k_bbox_tris<<<kPrimGrid, 256, 0, s>>>(tri_xyz, n, acc);
  emrt::note_launch(), k_bbox_fin<<<1, 32, 0, s>>>(acc, bbox);
}

}  // namespace emrt
