// Discovery (shoot-and-bounce with reception spheres) and image-method
// acceptance kernels.
#include <cfloat>

#include <cstring>

#include "trace.cuh"
#include "traverse.cuh"

namespace emrt {

namespace {

constexpr int kBounceBlock = 128;

// ----------------------------------------------------------------------------
// primary directions: Fibonacci sphere, z = 1 - (2i+1)/N, golden-angle
// azimuth, evaluated in double precision and rounded once to float32
__device__ inline float3 fib_dir(uint64_t n, uint64_t i) {
  double z = 1.0 - (2.0 * (double)i + 1.0) / (double)n;
  double rho = sqrt(fmax(0.0, 1.0 - z * z));
  double g = (3.0 - sqrt(5.0)) / 2.0;
  double t = (double)i * g;
  double phi = 2.0 * 3.14159265358979323846 * (t - floor(t));
  double sp, cp;
  sincos(phi, &sp, &cp);
  return make_float3((float)(rho * cp), (float)(rho * sp), (float)z);
}

// octahedral direction code: 16 bits per axis, interleaved
__device__ inline uint32_t spread16(uint32_t x) {
  x &= 0xffffu;
  x = (x | (x << 8)) & 0x00ff00ffu;
  x = (x | (x << 4)) & 0x0f0f0f0fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}
__device__ inline uint32_t oct_code(float3 d) {
  float s = fabsf(d.x) + fabsf(d.y) + fabsf(d.z);
  float u = d.x / s, v = d.y / s;
  if (d.z < 0.f) {
    float uu = (1.f - fabsf(v)) * (u >= 0.f ? 1.f : -1.f);
    float vv = (1.f - fabsf(u)) * (v >= 0.f ? 1.f : -1.f);
    u = uu;
    v = vv;
  }
  uint32_t a = (uint32_t)fminf(fmaxf((u * 0.5f + 0.5f) * 65535.f, 0.f), 65535.f);
  uint32_t b = (uint32_t)fminf(fmaxf((v * 0.5f + 0.5f) * 65535.f, 0.f), 65535.f);
  return spread16(a) << 1 | spread16(b);
}

__global__ void k_dir_codes(uint64_t n, uint64_t off, uint64_t stride, uint32_t count,
                            KeyW<1> *keys, uint32_t *vals) {
  uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= count) return;
  float3 d = fib_dir(n, off + stride * (uint64_t)j);
  keys[j].w[0] = oct_code(d);
  vals[j] = j;
}

__global__ void k_dir_table(uint64_t n, uint64_t off, uint64_t stride, uint32_t count,
                            const uint32_t *order, float4 *table) {
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  uint32_t j = order[k];
  float3 d = fib_dir(n, off + stride * (uint64_t)j);
  table[k] = make_float4(d.x, d.y, d.z, __uint_as_float(j));
}

// ----------------------------------------------------------------------------
__device__ inline uint32_t spread7(uint32_t v) {  // 7 bits -> every third bit
  uint32_t x = v & 0x7fu;
  x = (x | (x << 8)) & 0x0000f00fu;
  x = (x | (x << 4)) & 0x000c30c3u;
  x = (x | (x << 2)) & 0x00249249u;
  return x;
}

// Coherence cell of a ray: 7-bit-per-axis Morton code of its origin in the
// scene box and its 32-bit octahedral direction code.
__device__ inline void ray_cell(float3 o, float3 d, float4 lo, float4 hi, uint32_t &m,
                                uint32_t &oc) {
  uint32_t c[3];
  float q[3] = {(o.x - lo.x) / (hi.x - lo.x), (o.y - lo.y) / (hi.y - lo.y), (o.z - lo.z) / (hi.z - lo.z)};
  for (int k = 0; k < 3; k++) c[k] = (uint32_t)(fminf(fmaxf(q[k], 0.f), 1.f) * 127.f);
  m = spread7(c[0]) << 2 | spread7(c[1]) << 1 | spread7(c[2]);
  oc = oct_code(d);
}
// single-scene coherence key (24 bits): 5-bit-per-axis origin cell, 9-bit
// direction bin
__device__ inline uint32_t ray_key(float3 o, float3 d, float4 lo, float4 hi) {
  uint32_t m, oc;
  ray_cell(o, d, lo, hi, m, oc);
  return (m >> 6) << 9 | oc >> 23;
}

// ----------------------------------------------------------------------------
#include "bounce.cuh"
#include "chain.cuh"

// ----------------------------------------------------------------------------
// canonical key: tx | rx | depth | f0 | .. | f_{K-1}, most significant first
struct U128 { unsigned long long hi, lo; };
__device__ inline void push_bits(U128 &k, uint64_t v, int nb) {
  if (nb == 0) return;
  k.hi = (k.hi << nb) | (nb < 64 ? (k.lo >> (64 - nb)) : k.lo);
  k.lo = (nb < 64) ? ((k.lo << nb) | v) : v;
}

// canonical key of the record at r
__device__ inline KeyW<4> record_key(const uint32_t *r, const KeyLayout &kl) {
  const uint4 *q4 = reinterpret_cast<const uint4 *>(r);
  uint4 a = q4[0], b = q4[1];
  uint32_t depth = a.z & 15u;
  uint32_t f[4] = {a.w, b.x, b.y, b.z};
  U128 k = {0ull, 0ull};
  push_bits(k, a.x >> 8, kl.bs);   // scene (batched records; 0 bits otherwise)
  push_bits(k, a.x & 255u, kl.bt);
  push_bits(k, a.y, kl.br);
  push_bits(k, depth, 3);
  for (int q = 0; q < kl.K; q++) push_bits(k, q < (int)depth ? f[q] : 0u, kl.bf);
  KeyW<4> kk;
  kk.w[0] = (uint32_t)k.lo;
  kk.w[1] = (uint32_t)(k.lo >> 32);
  kk.w[2] = (uint32_t)k.hi;
  kk.w[3] = (uint32_t)(k.hi >> 32);
  return kk;
}

__global__ void k_path_keys(const uint32_t *rec, const uint32_t *n, uint32_t cap, KeyLayout kl,
                            KeyW<4> *keys, uint32_t *vals, uint32_t *n_eff) {
  uint32_t cnt = min(*n, cap);
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *n_eff = cnt;
  for (; i < cnt; i += gridDim.x * blockDim.x) {
    keys[i] = record_key(rec + 8ull * i, kl);
    vals[i] = i;
  }
}

__device__ inline bool key_eq(const KeyW<4> &a, const KeyW<4> &b) {
  return a.w[0] == b.w[0] && a.w[1] == b.w[1] && a.w[2] == b.w[2] && a.w[3] == b.w[3];
}

__device__ inline bool key_lt(const KeyW<4> &a, const KeyW<4> &b) {
  for (int q = 3; q >= 0; q--)
    if (a.w[q] != b.w[q]) return a.w[q] < b.w[q];
  return false;
}

// Stable merge of two runs of canonical keys, A = keys[0, na) and
// B = keys[na, n) with na = min(*na_p, cap_a, n), A first among equal keys.
// Output position k takes the element chosen after the binary search for the
// number of A keys among the first k outputs (the merge path).  A pair of
// neighbours out of order in A or in B raises ERR_UNSORTED.
__global__ void k_merge_path(const KeyW<4> *keys, const uint32_t *vals, const uint32_t *na_p,
                             uint32_t cap_a, const uint32_t *n_p, KeyW<4> *kout, uint32_t *vout,
                             Counters *ctr) {
  const uint32_t n = *n_p;
  const uint32_t na = min(min(*na_p, cap_a), n), nb = n - na;
  const KeyW<4> *A = keys, *B = keys + na;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    if (k < na ? (k > 0 && key_lt(A[k], A[k - 1]))
               : (k > na && key_lt(B[k - na], B[k - na - 1])))
      atomicOr(&ctr->err, ERR_UNSORTED);
    uint32_t lo = k > nb ? k - nb : 0, hi = min(k, na);
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (!key_lt(B[k - 1 - mid], A[mid])) lo = mid + 1;  // A[mid] precedes B[k-1-mid]
      else hi = mid;
    }
    const uint32_t i = lo, j = k - lo;
    const bool take_a = i < na && (j >= nb || !key_lt(B[j], A[i]));
    kout[k] = take_a ? A[i] : B[j];
    vout[k] = take_a ? vals[i] : vals[na + j];
  }
}

// equal keys above bit lb
__device__ inline bool key_prefix_eq(const KeyW<4> &a, const KeyW<4> &b, int lb) {
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int lo = 32 * q;
    if (lo + 32 <= lb) continue;
    const int sh = lb > lo ? lb - lo : 0;
    if ((a.w[q] >> sh) != (b.w[q] >> sh)) return false;
  }
  return true;
}

// Completes a sort ordered by the key bits from lb up: each run of keys equal
// in those bits is sorted by the whole key, in place, by the thread at its
// head (insertion sort for short runs, heap sort for long ones; the order of
// equal keys is not kept).
__global__ void k_sort_runs(KeyW<4> *k, uint32_t *v, const uint32_t *n, int lb) {
  const uint32_t cnt = *n;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    if (i > 0 && key_prefix_eq(k[i], k[i - 1], lb)) continue;
    uint32_t e = i + 1;
    while (e < cnt && key_prefix_eq(k[e], k[i], lb)) e++;
    const uint32_t len = e - i;
    if (len < 2) continue;
    KeyW<4> *kk = k + i;
    uint32_t *vv = v + i;
    if (len <= 32) {
      for (uint32_t a = 1; a < len; a++) {
        const KeyW<4> x = kk[a];
        const uint32_t xv = vv[a];
        uint32_t b = a;
        while (b > 0 && key_lt(x, kk[b - 1])) {
          kk[b] = kk[b - 1];
          vv[b] = vv[b - 1];
          b--;
        }
        kk[b] = x;
        vv[b] = xv;
      }
      continue;
    }
    auto swap = [&](uint32_t a, uint32_t b) {
      const KeyW<4> t = kk[a];
      kk[a] = kk[b];
      kk[b] = t;
      const uint32_t tv = vv[a];
      vv[a] = vv[b];
      vv[b] = tv;
    };
    auto sift = [&](uint32_t root, uint32_t end) {
      while (2 * root + 1 < end) {
        uint32_t c = 2 * root + 1;
        if (c + 1 < end && key_lt(kk[c], kk[c + 1])) c++;
        if (!key_lt(kk[root], kk[c])) break;
        swap(root, c);
        root = c;
      }
    };
    for (uint32_t r = len / 2; r-- > 0;) sift(r, len);
    for (uint32_t end = len - 1; end > 0; end--) {
      swap(0, end);
      sift(0, end);
    }
  }
}

// Candidates already in the cache: for each of the *n unique candidates (in
// canonical order) a binary search of the cache's canonical records;
// flag[i] = 1 for a candidate the cache does not hold.  A candidate the
// cache holds as a valid path lowers that record's smallest ray index to its
// own (what merging the accepted candidate would have done; one candidate per
// record, so no two threads write the same word).
__global__ void k_known(const uint32_t *cand, const uint32_t *n, uint32_t *cache,
                        const uint32_t *cache_n, uint32_t cache_cap, KeyLayout kl,
                        uint32_t *flag) {
  const uint32_t cnt = *n, nc = min(*cache_n, cache_cap);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    const KeyW<4> k = record_key(cand + 8ull * i, kl);
    uint32_t lo = 0, hi = nc;
    while (lo < hi) {  // first cache record whose key is not below k
      const uint32_t mid = (lo + hi) >> 1;
      if (key_lt(record_key(cache + 8ull * mid, kl), k)) lo = mid + 1;
      else hi = mid;
    }
    const bool found = lo < nc && key_eq(record_key(cache + 8ull * lo, kl), k);
    flag[i] = found ? 0u : 1u;
    if (found && (cache[8ull * lo + 2] & EMRT_PATH_VALID))
      cache[8ull * lo + 7] = min(cache[8ull * lo + 7], cand[8ull * i + 7]);
  }
}

// out[k] = rec[vals[k]] for k < min(*n, cap); ERR_PATH_OVERFLOW when *n > cap.
__global__ void k_gather_records(const uint32_t *rec, const uint32_t *vals, const uint32_t *n,
                                 uint32_t *out, uint32_t cap, Counters *ctr) {
  const uint32_t cnt = *n;
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && cnt > cap) atomicOr(&ctr->err, ERR_PATH_OVERFLOW);
  for (; i < min(cnt, cap); i += gridDim.x * blockDim.x) {
    const uint4 *r = reinterpret_cast<const uint4 *>(rec + 8ull * vals[i]);
    uint4 *o = reinterpret_cast<uint4 *>(out + 8ull * i);
    o[0] = r[0];
    o[1] = r[1];
  }
}

__global__ void k_heads(const KeyW<4> *keys, const uint32_t *n, uint32_t *head) {
  uint32_t cnt = *n;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
    head[i] = (i == 0 || !key_eq(keys[i], keys[i - 1])) ? 1u : 0u;
}

__global__ void k_unique(const uint32_t *rec, const KeyW<4> *keys, const uint32_t *vals,
                         const uint32_t *head, const uint32_t *pos, const uint32_t *n,
                         uint32_t *uniq) {
  uint32_t cnt = *n;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    if (!head[i]) continue;
    const uint4 *r = reinterpret_cast<const uint4 *>(rec + 8ull * vals[i]);
    uint4 a = r[0], b = r[1];
    uint32_t ray = b.w;
    for (uint32_t k = i + 1; k < cnt && !head[k]; k++) {
      uint32_t rj = rec[8ull * vals[k] + 7];
      ray = min(ray, rj);
    }
    b.w = ray;  // flags of the first record of the run are kept
    uint4 *o = reinterpret_cast<uint4 *>(uniq + 8ull * pos[i]);
    o[0] = a;
    o[1] = b;
  }
}

// ----------------------------------------------------------------------------
// image method in double precision
__device__ inline void plane_of(const GeomView &g, uint32_t f, D3 &n, double &d) {
  if (f < g.n_static_faces) {
    double4_32a p = g.face_plane[f];
    n = mkd(p.x, p.y, p.z);
    d = p.w;
    return;
  }
  uint32_t v = (f - g.n_static_faces) / 6u, j = (f - g.n_static_faces) % 6u;
  int ax = j >> 1;
  bool neg = (j & 1u) == 0;
  float4 lo = g.veh_lo[v], hi = g.veh_hi[v];
  double s = neg ? -1.0 : 1.0;
  n = mkd(ax == 0 ? s : 0.0, ax == 1 ? s : 0.0, ax == 2 ? s : 0.0);
  double c = ax == 0 ? (neg ? lo.x : hi.x) : (ax == 1 ? (neg ? lo.y : hi.y) : (neg ? lo.z : hi.z));
  d = s * c;
}

// signed distance of P (on the face plane) to the face boundary, >= 0 inside
__device__ inline double inface_margin(const GeomView &g, uint32_t f, D3 P, D3 n) {
  if (f < g.n_static_faces) {
    uint4 info = g.face_info[f];
    double m = 1e300;
    float4 a4 = g.face_vert[info.x + info.y - 1];
    D3 a = mkd(a4.x, a4.y, a4.z);
    for (uint32_t k = 0; k < info.y; k++) {
      float4 b4 = g.face_vert[info.x + k];
      D3 b = mkd(b4.x, b4.y, b4.z);
      D3 e = b - a;
      double sd = dotd(crossd(e, P - a), n) / normd(e);
      m = fmin(m, sd);
      a = b;
    }
    return m;
  }
  uint32_t v = (f - g.n_static_faces) / 6u, j = (f - g.n_static_faces) % 6u;
  int ax = j >> 1;
  float4 lo = g.veh_lo[v], hi = g.veh_hi[v];
  double p[3] = {P.x, P.y, P.z};
  double l[3] = {lo.x, lo.y, lo.z}, h[3] = {hi.x, hi.y, hi.z};
  double m = 1e300;
  for (int k = 0; k < 3; k++) {
    if (k == ax) continue;
    m = fmin(m, fmin(p[k] - l[k], h[k] - p[k]));
  }
  return m;
}

constexpr double kMargin = 1e-4;

// Acceptance runs in two phases so that the occlusion legs, long any-hit
// traversals, get a thread each.  Phase 1, per record: images across the
// face planes, reflection points backward from the receiver (FP64), the
// parameter and in-face tests with their margin; writes the depth and the
// geometric verdict to w2 and the k + 2 points, rounded to float32, to
// pts[p * cap + i].  Phase 2, per (leg q, record i), leg-major: any-hit test
// of the segment Q[q] -> Q[q+1] over static triangles and vehicle boxes with
// the endpoint faces excluded; an occluded leg clears EMRT_PATH_VALID.
template <bool BATCH>
__global__ void __launch_bounds__(kBounceBlock) k_accept_geom(GeomView G, const BatchScene *__restrict__ tab,
                                                              uint32_t *rec, const uint32_t *n,
                                                              float4 *pts, uint32_t cap) {
  __shared__ uint32_t s_cnt[EMRT_MAX_DEPTH + 2];
  __shared__ uint32_t s_order[kBounceBlock];
  const uint32_t cnt = min(*n, cap);
  // FP64 work per path grows with its depth: paths handed out by depth
  for (uint32_t base = blockIdx.x * blockDim.x; base < cnt; base += gridDim.x * blockDim.x) {
    const uint32_t i = depth_ordered(rec, base, cnt, s_cnt, s_order);
    if (i >= cnt) continue;
    uint4 *r = reinterpret_cast<uint4 *>(rec + 8ull * i);
    uint4 a = r[0], b = r[1];
    uint32_t k = a.z & 15u;
    uint32_t f[EMRT_MAX_DEPTH] = {a.w, b.x, b.y, b.z};
    const uint32_t sc = BATCH ? (a.x >> 8) : 0u, tx = BATCH ? (a.x & 255u) : a.x;
    const GeomView &g = BATCH ? tab[sc].g : G;
    bool ok = k <= EMRT_MAX_DEPTH && tx < g.n_tx && a.y < g.n_rx;
    uint32_t nf = g.n_static_faces + 6u * g.n_veh;
    for (uint32_t q = 0; ok && q < k; q++) ok = f[q] < nf && (q == 0 || f[q] != f[q - 1]);
    bool marg = false;
    if (ok) {
      D3 Q[EMRT_MAX_DEPTH + 2];
      D3 I[EMRT_MAX_DEPTH + 1];
      D3 nn[EMRT_MAX_DEPTH];
      double dd[EMRT_MAX_DEPTH];
      I[0] = tod(f3(g.tx_pos[tx]));
      for (uint32_t q = 0; q < k; q++) {
        plane_of(g, f[q], nn[q], dd[q]);
        I[q + 1] = I[q] - nn[q] * (2.0 * (dotd(nn[q], I[q]) - dd[q]));
      }
      Q[0] = I[0];
      Q[k + 1] = tod(f3(g.rx_pos[a.y]));
      for (int q = (int)k; q >= 1 && ok; q--) {
        D3 D = Q[q + 1] - I[q];
        double den = dotd(nn[q - 1], D);
        if (den == 0.0) { ok = false; break; }
        double t = (dd[q - 1] - dotd(nn[q - 1], I[q])) / den;
        if (!(t > 0.0 && t < 1.0)) { ok = false; break; }
        Q[q] = I[q] + D * t;
        double m = inface_margin(g, f[q - 1], Q[q], nn[q - 1]);
        if (m < 0.0) ok = false;
        if (fabs(m) < kMargin) marg = true;
      }
      if (ok)
        for (uint32_t q = 0; q <= k + 1; q++)
          pts[(uint64_t)q * cap + i] = make_float4((float)Q[q].x, (float)Q[q].y, (float)Q[q].z, 0.f);
    }
    const uint32_t flags = (ok ? EMRT_PATH_VALID : 0u) | (marg ? EMRT_PATH_MARGINAL : 0u);
    a.z = (a.z & 15u) | flags;
    r[0] = a;
  }
}

// Each leg's any-hit test is split over kOcclPieces threads, each taking
// one piece of t in (0, 1) on the same ray (so every t is the one the whole
// leg would compute): the leg is occluded iff some piece is.  The launch is
// latency-bound -- a few long legs (first legs from a transmitter across
// the city) kept most SMs idle -- and shorter pieces visit fewer nodes one
// after another.  Measured on the city frame (acceptance stage): 1 piece
// 0.22 ms, 2 0.20, 4 0.17, 8 0.17, 16 0.20; the same records.
constexpr uint32_t kOcclPieces = 4;
template <bool BATCH>
__global__ void __launch_bounds__(kBounceBlock) k_accept_occl(GeomView G, const BatchScene *__restrict__ tab,
                                                              uint32_t *rec, const uint32_t *n,
                                                              const float4 *pts, uint32_t cap,
                                                              Counters *ctr) {
  StackSlot stk[kStack];
  TravStats st;
  const uint32_t cnt = min(*n, cap);
  const uint32_t NO = EMRT_NO_FACE;
  unsigned long long occl = 0;
  const uint64_t items = (uint64_t)(EMRT_MAX_DEPTH + 1) * cnt * kOcclPieces;
  for (uint64_t it = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; it < items;
       it += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t piece = (uint32_t)(it % kOcclPieces);
    const uint64_t leg = it / kOcclPieces;
    const uint32_t q = (uint32_t)(leg / cnt), i = (uint32_t)(leg - (uint64_t)q * cnt);
    const uint4 *r = reinterpret_cast<const uint4 *>(rec + 8ull * i);
    const uint4 a = r[0];
    const uint32_t k = a.z & 15u;
    if (q > k || !(a.z & EMRT_PATH_VALID)) continue;
    const uint4 b = r[1];
    const uint32_t f[EMRT_MAX_DEPTH] = {a.w, b.x, b.y, b.z};
    const uint32_t sc = BATCH ? (a.x >> 8) : 0u;
    const GeomView &g = BATCH ? tab[sc].g : G;
    const float3 A = f3(pts[(uint64_t)q * cap + i]), B = f3(pts[(uint64_t)(q + 1) * cap + i]);
    const uint32_t e0 = q >= 1 ? f[q - 1] : NO, e1 = q < k ? f[q] : NO;
    const uint32_t v0 = (e0 != NO && e0 >= g.n_static_faces) ? (e0 - g.n_static_faces) / 6u : NO;
    const uint32_t v1 = (e1 != NO && e1 >= g.n_static_faces) ? (e1 - g.n_static_faces) / 6u : NO;
    RayQ rq;
    ray_setup(rq, A, B - A);
    // this piece's share of t in (0, 1); neighbouring pieces overlap by a
    // relative 2^-20 so that a hit exactly at a boundary falls in one of them
    const float hi = piece + 1u == kOcclPieces ? 1.f : (float)(piece + 1u) / kOcclPieces;
    const float lo = piece == 0u ? 0.f : (float)piece / kOcclPieces * (1.f - 9.5367431640625e-7f);
    float tmax = hi;
    uint32_t hf = NO;
    occl++;
    bool hit = trace_tris<true>(g.stat, rq, lo, tmax, hf, e0, e1, stk, st);
    tmax = hi;
    if (!hit) hit = trace_boxes<true>(g.dyn, rq, lo, tmax, hf, g.n_static_faces, v0, v1, stk, st);
    if (hit) atomicAnd(&rec[8ull * i + 2], ~EMRT_PATH_VALID);
  }
  add_u64(&ctr->occl_rays, occl);
  if (st.overflow) atomicOr(&ctr->err, ERR_STACK);
}

__global__ void k_keep_flags(const uint32_t *rec, const uint32_t *n, int keep_all, uint32_t *flag) {
  uint32_t cnt = *n;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
    flag[i] = (keep_all || (rec[8ull * i + 2] & EMRT_PATH_VALID)) ? 1u : 0u;
}

__global__ void k_scatter_rec(const uint32_t *in, const uint32_t *n, const uint32_t *flag,
                              const uint32_t *pos, uint32_t *out, uint32_t cap,
                              const uint32_t *total, Counters *ctr) {
  uint32_t cnt = *n;
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && *total > cap) atomicOr(&ctr->err, ERR_PATH_OVERFLOW);
  for (; i < cnt; i += gridDim.x * blockDim.x) {
    if (!flag[i]) continue;
    uint32_t p = pos[i];
    if (p >= cap) continue;
    const uint4 *s = reinterpret_cast<const uint4 *>(in + 8ull * i);
    uint4 *d = reinterpret_cast<uint4 *>(out + 8ull * p);
    d[0] = s[0];
    d[1] = s[1];
  }
}

__global__ void k_copy_rec(const uint32_t *in, const uint32_t *n, uint32_t *out, uint32_t cap) {
  uint32_t cnt = min(*n, cap);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    const uint4 *s = reinterpret_cast<const uint4 *>(in + 8ull * i);
    uint4 *d = reinterpret_cast<uint4 *>(out + 8ull * i);
    d[0] = s[0];
    d[1] = s[1];
  }
}

__global__ void k_concat(const uint32_t *a, const uint32_t *na, uint32_t cap_a, const uint32_t *b,
                         const uint32_t *nb, uint32_t cap_b, uint32_t *dst, uint32_t dst_cap,
                         uint32_t *n_dst, Counters *ctr) {
  uint32_t ca = min(*na, cap_a), cb = min(*nb, cap_b);
  uint32_t tot = ca + cb;
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *n_dst = min(tot, dst_cap);
    if (tot > dst_cap) atomicOr(&ctr->err, ERR_CAND_OVERFLOW);
  }
  for (; i < min(tot, dst_cap); i += gridDim.x * blockDim.x) {
    const uint4 *s = reinterpret_cast<const uint4 *>(i < ca ? a + 8ull * i : b + 8ull * (i - ca));
    uint4 *d = reinterpret_cast<uint4 *>(dst + 8ull * i);
    d[0] = s[0];
    d[1] = s[1];
  }
}

__global__ void k_set_u32(uint32_t *p, uint32_t v) { *p = v; }

__global__ void k_gather_points(const float4 *pos, const uint32_t *ids, uint32_t n, float4 *out) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = pos[ids[i]];
}

__global__ void k_reverse_cand(uint32_t *cand, const uint32_t *n, uint32_t cap,
                               const uint32_t *ids) {
  const uint32_t cnt = min(*n, cap);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    uint4 *c = reinterpret_cast<uint4 *>(cand + 8ull * i);
    uint4 a = c[0], b = c[1];
    const uint32_t depth = a.z & 15u;
    const uint32_t f[EMRT_MAX_DEPTH] = {a.w, b.x, b.y, b.z};
    uint32_t r[EMRT_MAX_DEPTH];
#pragma unroll
    for (int k = 0; k < EMRT_MAX_DEPTH; k++)
      r[k] = (uint32_t)k < depth ? f[depth - 1 - k] : EMRT_NO_FACE;
    c[0] = make_uint4(a.y, ids ? ids[a.x] : a.x, a.z, r[0]);
    c[1] = make_uint4(r[1], r[2], r[3], b.w);
  }
}

__global__ void k_batch_first(const uint32_t *rec, const uint32_t *n, const uint32_t *flag,
                              const uint32_t *pos, uint32_t *first, uint32_t *cnt) {
  uint32_t c = *n;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < c; i += gridDim.x * blockDim.x) {
    if (!flag[i]) continue;
    uint32_t sc = rec[8ull * i] >> 8;
    if (sc >= kBatchMaxScenes) continue;
    atomicMin(&first[sc], pos[i]);
    atomicAdd(&cnt[sc], 1u);
  }
}

__global__ void k_batch_write(const BatchScene *tab, uint32_t n_scenes, const uint32_t *rec,
                              const uint32_t *n, const uint32_t *flag, const uint32_t *pos,
                              const uint32_t *first, const uint32_t *cnt, Counters *ctr) {
  uint32_t c = *n;
  uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_scenes) {
    *tab[t].out_count = cnt[t];
    if (cnt[t] > tab[t].out_cap) atomicOr(&ctr->err, ERR_PATH_OVERFLOW);
  }
  for (uint32_t i = t; i < c; i += gridDim.x * blockDim.x) {
    if (!flag[i]) continue;
    const uint4 *src = reinterpret_cast<const uint4 *>(rec + 8ull * i);
    uint4 a = src[0], b = src[1];
    uint32_t sc = a.x >> 8;
    if (sc >= n_scenes) continue;
    uint32_t p = pos[i] - first[sc];
    if (p >= tab[sc].out_cap) continue;
    a.x &= 255u;
    uint4 *dst = reinterpret_cast<uint4 *>(tab[sc].out_rec + 8ull * p);
    dst[0] = a;
    dst[1] = b;
  }
}

__global__ void k_batch_init(uint32_t *first, uint32_t *cnt) {
  uint32_t t = threadIdx.x;
  if (t < kBatchMaxScenes) {
    first[t] = 0xffffffffu;
    cnt[t] = 0u;
  }
}

__global__ void k_ray_keys(const Ray *r, const uint32_t *n, const float4 *bb, KeyW<1> *keys,
                           uint32_t *vals, bool batched) {
  uint32_t cnt = *n;
  float4 lo = bb[0], hi = bb[1];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    float4 o = r[i].o_L, d = r[i].d_id;
    uint32_t m, oc;
    ray_cell(f3(o), f3(d), lo, hi, m, oc);
    keys[i].w[0] = batched ? ((__float_as_uint(d.w) >> 26) << 18 | (m >> 9) << 6 | oc >> 26)
                           : ((m >> 6) << 9 | oc >> 23);
    vals[i] = i;
  }
}

int g_bounce_grid = 0;

}  // namespace

KeyLayout key_layout(uint32_t n_tx, uint32_t n_rx, uint32_t n_faces, int K, uint32_t n_scenes) {
  auto bits = [](uint32_t v) {  // bits to hold 0..v-1
    int b = 0;
    while (b < 32 && (1ull << b) < (unsigned long long)v) b++;
    return b;
  };
  KeyLayout kl;
  kl.bs = n_scenes > 1 ? bits(n_scenes) : 0;
  kl.bt = bits(n_tx);
  kl.br = bits(n_rx);
  kl.bf = bits(n_faces);
  kl.K = K;
  kl.total = kl.bs + kl.bt + kl.br + 3 + K * kl.bf;
  return kl;
}

int g_chain_grid = 0;
int chain_grid() {
  if (!g_chain_grid) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_chain<kBounceBlock>, kBounceBlock, 0);
    g_chain_grid = sms * (per > 0 ? per : 1);
  }
  return g_chain_grid;
}

uint64_t chain_queue_entries() {
  return (uint64_t)chain_grid() * (kBounceBlock / 32) * kChainQueue;
}

void launch_chain(const BounceLaunch &L, const ChainBufs &D, int grid, cudaStream_t s) {
  emrt::note_launch(), k_chain<kBounceBlock><<<grid, kBounceBlock, 0, s>>>(L, D);
}

int g_walk_grid[2] = {0, 0};
template <bool WIDE>
int walk_grid() {
  if (!g_walk_grid[WIDE]) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_walk<kBounceBlock, false, WIDE>,
                                                  kBounceBlock, 0);
    g_walk_grid[WIDE] = sms * (per > 0 ? per : 1);
  }
  return g_walk_grid[WIDE];
}

void launch_walk(const BounceLaunch &L, cudaStream_t s, bool wide) {
  if (wide)
    emrt::note_launch(), k_walk<kBounceBlock, false, true><<<walk_grid<true>(), kBounceBlock, 0, s>>>(L, nullptr, 1);
  else
    emrt::note_launch(), k_walk<kBounceBlock, false><<<walk_grid<false>(), kBounceBlock, 0, s>>>(L, nullptr, 1);
}

void launch_tx_epoch(const float4 *pos, float4 *ref, uint32_t *epoch, uint32_t n_tx,
                     cudaStream_t s) {
  emrt::note_launch(), k_tx_epoch<<<ceil_div(n_tx, 64), 64, 0, s>>>(pos, ref, epoch, n_tx);
}

int bounce_grid() {
  if (!g_bounce_grid) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bounce<false, kBounceBlock, 32, false>,
                                                  kBounceBlock, 0);
    g_bounce_grid = sms * (per > 0 ? per : 1);
  }
  return g_bounce_grid;
}

namespace {
struct Variant {
  const char *name;
  int block;
  void (*kern)(BounceLaunch, const BatchScene *, uint32_t);
  bool walk;  // depth-first: one launch for all bounces
  int grid;
};
Variant g_variants[] = {
    {"block64_fetch32", 64, k_bounce<true, 64, 32, false>, false, 0},
    {"block128_fetch32", 128, k_bounce<true, 128, 32, false>, false, 0},
    {"block256_fetch32", 256, k_bounce<true, 256, 32, false>, false, 0},
    {"block128_fetch128", 128, k_bounce<true, 128, 128, false>, false, 0},
    {"block256_fetch64", 256, k_bounce<true, 256, 64, false>, false, 0},
    {"block64_fetch128", 64, k_bounce<true, 64, 128, false>, false, 0},
    {"block128_fetch32_bvh8", 128, k_bounce<true, 128, 32, true>, false, 0},
    {"block64_fetch32_bvh8", 64, k_bounce<true, 64, 32, true>, false, 0},
    {"depth_first_block128", 128, k_walk<128, true>, true, 0},
    {"depth_first_block64", 64, k_walk<64, true>, true, 0},
    {"depth_first_block256", 256, k_walk<256, true>, true, 0},
    {"depth_first_block128_bvh8", 128, k_walk<128, true, true>, true, 0},
};
constexpr int kNumVariants = sizeof(g_variants) / sizeof(g_variants[0]);
}  // namespace

int n_bounce_variants() { return kNumVariants; }
const char *bounce_variant_name(int v) { return g_variants[v].name; }
bool bounce_variant_depth_first(int v) { return g_variants[v].walk; }
int variant_named(const char *name) {
  for (int v = 0; v < kNumVariants; v++)
    if (!strcmp(g_variants[v].name, name)) return v;
  return 0;
}
// fastest on the 64-scene batch measured, of either form
int default_bounce_variant() { return variant_named("depth_first_block128"); }
int default_breadth_first_variant() { return variant_named("block128_fetch32"); }
int bounce_variant_grid(int v) {
  Variant &V = g_variants[v];
  if (!V.grid) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, V.kern, V.block, 0);
    V.grid = sms * (per > 0 ? per : 1);
  }
  return V.grid;
}

void launch_bounce_batched(int variant, const BounceLaunch &L, const BatchScene *tab,
                           uint32_t n_scenes, cudaStream_t s) {
  Variant &V = g_variants[variant];
  emrt::note_launch(), V.kern<<<bounce_variant_grid(variant), V.block, 0, s>>>(L, tab, n_scenes);
}

void launch_accept_batched(const BatchScene *tab, uint32_t *rec, const uint32_t *n, Counters *ctr,
                           float4 *pts, uint32_t cap, cudaStream_t s) {
  GeomView none{};
  emrt::note_launch(), k_accept_geom<true><<<kPrimGrid * 4, kBounceBlock, 0, s>>>(none, tab, rec, n, pts, cap);
  emrt::note_launch(), k_accept_occl<true><<<kPrimGrid * 8, kBounceBlock, 0, s>>>(none, tab, rec, n, pts, cap, ctr);
}

void launch_batch_scatter(const BatchScene *tab, uint32_t n_scenes, const uint32_t *rec,
                          const uint32_t *n, const uint32_t *flag, const uint32_t *pos,
                          uint32_t *first, uint32_t *cnt, Counters *ctr, cudaStream_t s) {
  emrt::note_launch(), k_batch_init<<<1, kBatchMaxScenes, 0, s>>>(first, cnt);
  emrt::note_launch(), k_batch_first<<<kPrimGrid * 4, 256, 0, s>>>(rec, n, flag, pos, first, cnt);
  emrt::note_launch(), k_batch_write<<<kPrimGrid * 4, 256, 0, s>>>(tab, n_scenes, rec, n, flag, pos,
                                                                  first, cnt, ctr);
}

void build_dir_table(uint64_t n_rays, uint64_t offset, uint64_t stride, uint32_t count,
                     float4 *table, KeyW<1> *k0, KeyW<1> *k1, uint32_t *v0, uint32_t *v1,
                     uint32_t *d_n, uint32_t *hist, cudaStream_t s) {
  if (!count) return;
  emrt::note_launch(), k_dir_codes<<<ceil_div(count, 256), 256, 0, s>>>(n_rays, offset, stride, count, k0, v0);
  emrt::note_launch(), k_set_u32<<<1, 1, 0, s>>>(d_n, count);
  bool alt = radix_sort<1>(d_n, k0, v0, k1, v1, 32, hist, s, count);
  emrt::note_launch(), k_dir_table<<<ceil_div(count, 256), 256, 0, s>>>(n_rays, offset, stride, count, alt ? v1 : v0,
                                                   table);
}

void launch_ray_keys(const Ray *r, const uint32_t *n, const float4 *bbox, KeyW<1> *keys,
                     uint32_t *vals, cudaStream_t s, bool batched) {
  emrt::note_launch(), k_ray_keys<<<kPrimGrid * 8, 256, 0, s>>>(r, n, bbox, keys, vals, batched);
}

void launch_bounce(const BounceLaunch &L, int grid, cudaStream_t s, bool wide) {
  if (wide)
    emrt::note_launch(), k_bounce<false, kBounceBlock, 32, true><<<grid, kBounceBlock, 0, s>>>(L, nullptr, 1);
  else
    emrt::note_launch(), k_bounce<false, kBounceBlock, 32, false><<<grid, kBounceBlock, 0, s>>>(L, nullptr, 1);
}

void launch_path_keys(const uint32_t *rec, const uint32_t *n, uint32_t cap, KeyLayout kl,
                      KeyW<4> *keys, uint32_t *vals, uint32_t *n_eff, cudaStream_t s) {
  emrt::note_launch(), k_path_keys<<<kPrimGrid * 4, 256, 0, s>>>(rec, n, cap, kl, keys, vals, n_eff);
}
void launch_heads(const KeyW<4> *keys, const uint32_t *n, uint32_t *head, cudaStream_t s) {
  emrt::note_launch(), k_heads<<<kPrimGrid * 4, 256, 0, s>>>(keys, n, head);
}
void launch_unique(const uint32_t *rec, const KeyW<4> *keys, const uint32_t *vals,
                   const uint32_t *head, const uint32_t *pos, const uint32_t *n, uint32_t *uniq,
                   cudaStream_t s) {
  emrt::note_launch(), k_unique<<<kPrimGrid * 4, 256, 0, s>>>(rec, keys, vals, head, pos, n, uniq);
}
void launch_accept(const GeomView &g, uint32_t *rec, const uint32_t *n, Counters *ctr,
                   float4 *pts, uint32_t cap, cudaStream_t s) {
  emrt::note_launch(), k_accept_geom<false><<<kPrimGrid * 4, kBounceBlock, 0, s>>>(g, nullptr, rec, n, pts, cap);
  emrt::note_launch(), k_accept_occl<false><<<kPrimGrid * 8, kBounceBlock, 0, s>>>(g, nullptr, rec, n, pts, cap, ctr);
}
void launch_keep_flags(const uint32_t *rec, const uint32_t *n, int keep_all, uint32_t *flag,
                       cudaStream_t s) {
  emrt::note_launch(), k_keep_flags<<<kPrimGrid * 4, 256, 0, s>>>(rec, n, keep_all, flag);
}
void launch_scatter(const uint32_t *in, const uint32_t *n, const uint32_t *flag,
                    const uint32_t *pos, uint32_t *out, uint32_t cap, const uint32_t *total,
                    Counters *ctr, cudaStream_t s) {
  emrt::note_launch(), k_scatter_rec<<<kPrimGrid * 4, 256, 0, s>>>(in, n, flag, pos, out, cap, total, ctr);
}
void launch_copy_records(const uint32_t *in, const uint32_t *n, uint32_t *out, uint32_t cap,
                         cudaStream_t s) {
  emrt::note_launch(), k_copy_rec<<<kPrimGrid * 4, 256, 0, s>>>(in, n, out, cap);
}
void launch_concat(const uint32_t *a, const uint32_t *na, uint32_t cap_a, const uint32_t *b,
                   const uint32_t *nb, uint32_t cap_b, uint32_t *dst, uint32_t dst_cap,
                   uint32_t *n_dst, Counters *ctr, cudaStream_t s) {
  emrt::note_launch(), k_concat<<<kPrimGrid * 4, 256, 0, s>>>(a, na, cap_a, b, nb, cap_b, dst, dst_cap, n_dst, ctr);
}
void launch_merge_path(const KeyW<4> *keys, const uint32_t *vals, const uint32_t *na, uint32_t cap_a,
                       const uint32_t *n, KeyW<4> *kout, uint32_t *vout, Counters *ctr,
                       cudaStream_t s) {
  emrt::note_launch(), k_merge_path<<<kPrimGrid * 4, 256, 0, s>>>(keys, vals, na, cap_a, n, kout, vout, ctr);
}
void launch_known(const uint32_t *cand, const uint32_t *n, uint32_t *cache, const uint32_t *cache_n,
                  uint32_t cache_cap, KeyLayout kl, uint32_t *flag, cudaStream_t s) {
  emrt::note_launch(), k_known<<<kPrimGrid * 4, 256, 0, s>>>(cand, n, cache, cache_n, cache_cap, kl, flag);
}
void launch_gather_records(const uint32_t *rec, const uint32_t *vals, const uint32_t *n,
                           uint32_t *out, uint32_t cap, Counters *ctr, cudaStream_t s) {
  emrt::note_launch(), k_gather_records<<<kPrimGrid * 4, 256, 0, s>>>(rec, vals, n, out, cap, ctr);
}
void launch_sort_runs(KeyW<4> *keys, uint32_t *vals, const uint32_t *n, int low_bits,
                      cudaStream_t s) {
  emrt::note_launch(), k_sort_runs<<<kPrimGrid * 4, 256, 0, s>>>(keys, vals, n, low_bits);
}
void launch_set_u32(uint32_t *p, uint32_t v, cudaStream_t s) { emrt::note_launch(), k_set_u32<<<1, 1, 0, s>>>(p, v); }

void launch_gather_points(const float4 *pos, const uint32_t *ids, uint32_t n, float4 *out,
                          cudaStream_t s) {
  if (n) emrt::note_launch(), k_gather_points<<<ceil_div(n, 256), 256, 0, s>>>(pos, ids, n, out);
}
void launch_reverse_candidates(uint32_t *cand, const uint32_t *n, uint32_t cap,
                               const uint32_t *ids, cudaStream_t s) {
  emrt::note_launch(), k_reverse_cand<<<kPrimGrid * 4, 256, 0, s>>>(cand, n, cap, ids);
}

}  // namespace emrt
