// LBVH build and refit.  Binary radix tree of Karras (2012, "Maximizing
// parallelism in the construction of BVHs, octrees and k-d trees"), restated
// from the published algorithm; boxes are filled bottom-up with one arrival
// counter per inner node (the second thread to arrive merges the children).
#include <cfloat>

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

__device__ inline int delta(const KeyW<2> *k, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  uint64_t a = get_key(k[i]), b = get_key(k[j]);
  if (a == b) return 64 + __clz(i ^ j);
  return __clzll(a ^ b);
}

// one thread per inner node i in [0, n-2]
__global__ void k_hierarchy(const KeyW<2> *k, int n, float4 *nodes, uint32_t *leaf_parent) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int d = (delta(k, n, i, i + 1) - delta(k, n, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = delta(k, n, i, i - d);
  int lmax = 2;
  while (delta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(k, n, i, i + (l + t) * d) > dmin) l += t;
  int j = i + l * d;
  int dnode = delta(k, n, i, j);
  int s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (delta(k, n, i, i + (s + t) * d) > dnode) s += t;
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

// Bottom-up boxes: one thread per leaf walks to the root; the second child
// to arrive at a node continues.  MULTI: leaves of 1-4 prims (leaf code
// ~(first << 2 | count - 1)); prims other than a leaf's first have
// leaf_parent 0xFFFFFFFF.
template <int KIND, bool MULTI = false>
__global__ void k_refit(const float4 *prims, uint32_t n, float4 *nodes, const uint32_t *leaf_parent,
                        uint32_t *flags) {
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
  for (int guard = 0; guard < 4096; guard++) {  // tree depth bound (safety net)
    int p = code >> 1, side = code & 1;
    float4 *np = nodes + 4ll * p;
    reinterpret_cast<float4 *>(np + side)[0] = make_float4(b.lo.x, b.hi.x, b.lo.y, b.hi.y);
    reinterpret_cast<float2 *>(np + 2)[side] = make_float2(b.lo.z, b.hi.z);
    __threadfence();
    if (atomicAdd(&flags[p], 1u) == 0) return;
    __threadfence();
    float4 a0 = __ldcg(np), a1 = __ldcg(np + 1), a2 = __ldcg(np + 2);
    b.lo = make_float3(fminf(a0.x, a1.x), fminf(a0.z, a1.z), fminf(a2.x, a2.z));
    b.hi = make_float3(fmaxf(a0.y, a1.y), fmaxf(a0.w, a1.w), fmaxf(a2.y, a2.w));
    int pc = __ldcg(reinterpret_cast<const int *>(np + 3) + 2);
    if (pc < 0) return;
    code = pc;
  }
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

// one thread per 4-wide node of the current level
__global__ void k_collapse(const float4 *bn, const uint32_t *in_bin, const uint32_t *in_dst,
                           const uint32_t *n_in, float4 *out4, uint32_t *out_bin,
                           uint32_t *out_dst, uint32_t *n_out, uint32_t *n_alloc) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *n_in) return;
  int b = (int)in_bin[i];
  uint32_t dst = in_dst[i];
  Child c[4];
  int cnt = 2;
  c[0] = child_of(bn, b, 0);
  c[1] = child_of(bn, b, 1);
  while (cnt < 4) {
    int best = -1;
    float ba = -1.f;
    for (int k = 0; k < cnt; k++)
      if (c[k].code >= 0 && half_area(c[k]) > ba) {
        ba = half_area(c[k]);
        best = k;
      }
    if (best < 0) break;
    int nb = c[best].code;
    c[best] = child_of(bn, nb, 0);
    c[cnt++] = child_of(bn, nb, 1);
  }
  float4 *o = out4 + 8ull * dst;
  float v[6][4];
  int codes[4] = {0, 0, 0, 0};
  for (int k = 0; k < 4; k++) {
    bool ok = k < cnt;
    for (int a = 0; a < 3; a++) {
      v[2 * a][k] = ok ? c[k].lo[a] : 0.f;
      v[2 * a + 1][k] = ok ? c[k].hi[a] : 0.f;
    }
    if (!ok) continue;
    if (c[k].code < 0) {
      codes[k] = c[k].code;
    } else {
      uint32_t ni = atomicAdd(n_alloc, 1u);
      uint32_t slot = atomicAdd(n_out, 1u);
      out_bin[slot] = (uint32_t)c[k].code;
      out_dst[slot] = ni;
      codes[k] = (int)ni;
    }
  }
  for (int r = 0; r < 6; r++) o[r] = make_float4(v[r][0], v[r][1], v[r][2], v[r][3]);
  o[6] = make_float4(__int_as_float(codes[0]), __int_as_float(codes[1]), __int_as_float(codes[2]),
                     __int_as_float(codes[3]));
  o[7] = make_float4(__int_as_float(cnt), 0.f, 0.f, 0.f);
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

template <int KIND>
cudaError_t finish_build(BVHBuf &b, cudaStream_t s) {
  uint32_t n = b.n;
  if (n >= 2) {
    emrt::note_launch(), k_hierarchy<<<ceil_div(n - 1, 256), 256, 0, s>>>(b.keys, (int)n, b.nodes, b.leaf_parent);
    cudaMemsetAsync(b.flags, 0, sizeof(uint32_t) * n, s);
    emrt::note_launch(), k_refit<KIND><<<ceil_div(n, 256), 256, 0, s>>>(b.prims, n, b.nodes, b.leaf_parent, b.flags);
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
  v.nodes4 = nodes4;
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
  return e;
}

void bvh_free(BVHBuf &b) {
  cudaFree(b.nodes); cudaFree(b.prims); cudaFree(b.leaf_parent); cudaFree(b.flags);
  cudaFree(b.keys); cudaFree(b.keys2); cudaFree(b.idx); cudaFree(b.idx2); cudaFree(b.d_n);
  cudaFree(b.nodes4);
  b.nodes4 = nullptr;
  b.n4 = 0;
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

cudaError_t bvh_build_boxes(BVHBuf &b, const float4 *lo, const float4 *hi, uint32_t n,
                            const float4 *bbox, uint32_t *hist, cudaStream_t s) {
  b.n = n;
  if (n == 0) return cudaSuccess;
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
    emrt::note_launch(), k_refit<PRIM_BOX><<<ceil_div(n, 256), 256, 0, s>>>(b.prims, n, b.nodes, b.leaf_parent, b.flags);
  }
  return cudaGetLastError();
}

cudaError_t bvh_build_points(BVHBuf &b, const float4 *pts, uint32_t n, const float4 *bbox,
                             uint32_t *hist, cudaStream_t s) {
  b.n = n;
  if (n == 0) return cudaSuccess;
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
// ranges of up to this many triangles become leaves (1-4; on the city 1 is
// fastest: 4-triangle leaves cut node visits 29.0 -> 25.7 per segment but
// raised triangle tests 2.5 -> 6.7 and the traversal 16.0 -> 18.8 ms)
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
  uint32_t *tmp = nullptr, *ctr = nullptr;
  SahTask *tasks[2] = {nullptr, nullptr};
  if ((e = cudaMalloc(&cen, sizeof(float4) * n))) return e;
  if ((e = cudaMalloc(&lo, sizeof(float4) * n))) return e;
  if ((e = cudaMalloc(&hi, sizeof(float4) * n))) return e;
  if ((e = cudaMalloc(&tmp, sizeof(uint32_t) * n))) return e;
  if ((e = cudaMalloc(&tasks[0], sizeof(SahTask) * (n / 2 + 2)))) return e;
  if ((e = cudaMalloc(&tasks[1], sizeof(SahTask) * (n / 2 + 2)))) return e;
  if ((e = cudaMalloc(&ctr, sizeof(uint32_t) * 4))) return e;
  emrt::note_launch(), k_tri_bounds<<<ceil_div(n, 256), 256, 0, s>>>(tri_xyz, n, cen, lo, hi, b.idx);
  if (n >= 2) {
    SahTask root{0u, n, 0u, 0u};
    uint32_t init[4] = {1, 0, 1, 0};  // level sizes [0],[1]; nodes allocated [2]
    cudaMemcpyAsync(tasks[0], &root, sizeof(root), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(ctr, init, sizeof(init), cudaMemcpyHostToDevice, s);
    uint32_t n_level = 1, zero = 0;
    int cur = 0, levels = 0;
    for (; n_level && levels < kSahMaxDepth; levels++) {
      cudaMemcpyAsync(ctr + (cur ^ 1), &zero, sizeof(uint32_t), cudaMemcpyHostToDevice, s);
      emrt::note_launch(), k_sah_level<<<n_level, kSahBlock, 0, s>>>(
          tasks[cur], ctr + cur, cen, lo, hi, b.idx, tmp, b.nodes, b.leaf_parent, tasks[cur ^ 1],
          ctr + (cur ^ 1), ctr + 2);
      cudaMemcpyAsync(&n_level, ctr + (cur ^ 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
      if ((e = cudaStreamSynchronize(s))) break;
      cur ^= 1;
    }
    // a tree deeper than the traversal stack can serve is not used: the
    // caller falls back to the LBVH
    if (!e && n_level) e = cudaErrorNotSupported;
  }
  if (!e) {
    emrt::note_launch(), k_gather_tris<<<ceil_div(n, 256), 256, 0, s>>>(tri_xyz, tri_face, b.idx, n, b.prims);
    if (n >= 2) {
      cudaMemsetAsync(b.flags, 0, sizeof(uint32_t) * n, s);
      emrt::note_launch(), k_refit<PRIM_TRI, true><<<ceil_div(n, 256), 256, 0, s>>>(b.prims, n, b.nodes, b.leaf_parent, b.flags);
    }
    e = cudaStreamSynchronize(s);
    if (!e) b.leaf_bits = 2;
  }
  cudaFree(cen); cudaFree(lo); cudaFree(hi); cudaFree(tmp);
  cudaFree(tasks[0]); cudaFree(tasks[1]); cudaFree(ctr);
  if (e) return e;
  return cudaGetLastError();
}

cudaError_t bvh4_collapse(BVHBuf &b, cudaStream_t s) {
  if (b.n < 2) return cudaSuccess;
  cudaError_t e;
  cudaFree(b.nodes4);
  b.nodes4 = nullptr;
  if ((e = cudaMalloc(&b.nodes4, sizeof(float4) * 8 * (size_t)b.n))) return e;
  uint32_t *buf = nullptr;  // two level lists (binary index, 4-wide index) + counters
  if ((e = cudaMalloc(&buf, sizeof(uint32_t) * (4 * (size_t)b.n + 4)))) return e;
  uint32_t *lb[2] = {buf, buf + b.n}, *ld[2] = {buf + 2 * b.n, buf + 3 * b.n};
  uint32_t *ctr = buf + 4 * b.n;  // [0],[1]: level sizes, [2]: nodes allocated
  uint32_t init[4] = {1, 0, 1, 0};
  uint32_t zero = 0;
  cudaMemcpyAsync(ctr, init, sizeof(init), cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(lb[0], 0, sizeof(uint32_t), s);
  cudaMemsetAsync(ld[0], 0, sizeof(uint32_t), s);
  uint32_t n_level = 1;
  int cur = 0;
  for (int guard = 0; n_level && guard < 4096; guard++) {
    cudaMemcpyAsync(ctr + (cur ^ 1), &zero, sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    emrt::note_launch(), k_collapse<<<ceil_div(n_level, 128), 128, 0, s>>>(
        b.nodes, lb[cur], ld[cur], ctr + cur, b.nodes4, lb[cur ^ 1], ld[cur ^ 1], ctr + (cur ^ 1),
        ctr + 2);
    cudaMemcpyAsync(&n_level, ctr + (cur ^ 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) break;
    cur ^= 1;
  }
  cudaMemcpyAsync(&b.n4, ctr + 2, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  cudaFree(buf);
  if (e) return e;
  return cudaGetLastError();
}

void bbox_of_tris(const float *tri_xyz, uint32_t n, float4 *bbox, cudaStream_t s) {
  uint32_t *acc = reinterpret_cast<uint32_t *>(bbox + 2);  // 6 words of scratch after bbox
  emrt::note_launch(), k_bbox_init<<<1, 32, 0, s>>>(acc);
  if (n) emrt::note_launch(), k_bbox_tris<<<kPrimGrid, 256, 0, s>>>(tri_xyz, n, acc);
  emrt::note_launch(), k_bbox_fin<<<1, 32, 0, s>>>(acc, bbox);
}

}  // namespace emrt
