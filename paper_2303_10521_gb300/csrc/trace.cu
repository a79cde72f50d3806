// Discovery (shoot-and-bounce with reception spheres) and image-method
// acceptance kernels.
#include <cfloat>

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
__device__ inline float3 face_normal_f(const GeomView &g, uint32_t f) {
  if (f < g.n_static_faces) {
    double4 p = g.face_plane[f];
    return make_float3((float)p.x, (float)p.y, (float)p.z);
  }
  uint32_t j = (f - g.n_static_faces) % 6u;
  float s = (j & 1u) ? 1.f : -1.f;
  int ax = j >> 1;
  return make_float3(ax == 0 ? s : 0.f, ax == 1 ? s : 0.f, ax == 2 ? s : 0.f);
}

__device__ inline void rx_bounds(const BVHView &b, float3 &lo, float3 &hi) {
  if (b.n_prims >= 2) {
    float4 n0 = ldg4(b.nodes), n1 = ldg4(b.nodes + 1), n2 = ldg4(b.nodes + 2);
    lo = make_float3(fminf(n0.x, n1.x), fminf(n0.z, n1.z), fminf(n2.x, n2.z));
    hi = make_float3(fmaxf(n0.y, n1.y), fmaxf(n0.w, n1.w), fmaxf(n2.y, n2.w));
  } else if (b.n_prims == 1) {
    lo = hi = f3(ldg4(b.prims));
  } else {
    lo = hi = make_float3(0.f, 0.f, 0.f);
  }
}

__device__ inline void add_u64(unsigned long long *p, unsigned long long v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(p, v);
}

// Specular continuation of a segment that hit `face` at t: hit point p and
// mirrored unit direction r.  Explicit roundings, so that every kernel that
// continues a chain produces the same bits.
__device__ inline void reflect_step(const GeomView &g, uint32_t face, float3 o, float3 d, float t,
                                    float3 &p, float3 &r) {
  const float3 n = face_normal_f(g, face);
  p = make_float3(__fmaf_rn(d.x, t, o.x), __fmaf_rn(d.y, t, o.y), __fmaf_rn(d.z, t, o.z));
  const float dn = __fmul_rn(2.f, __fmaf_rn(d.z, n.z, __fmaf_rn(d.y, n.y, __fmul_rn(d.x, n.x))));
  r = make_float3(__fmaf_rn(-n.x, dn, d.x), __fmaf_rn(-n.y, dn, d.y), __fmaf_rn(-n.z, dn, d.z));
  const float inv = rsqrtf(__fmaf_rn(r.z, r.z, __fmaf_rn(r.y, r.y, __fmul_rn(r.x, r.x))));
  r = make_float3(__fmul_rn(r.x, inv), __fmul_rn(r.y, inv), __fmul_rn(r.z, inv));
}

// Escape distance of a ray that hit nothing: the furthest projection of the
// receiver bounds on the ray.
__device__ inline float escape_t(float3 o, float3 d, float3 rlo, float3 rhi) {
  return fmaxf(d.x * (rlo.x - o.x), d.x * (rhi.x - o.x)) +
         fmaxf(d.y * (rlo.y - o.y), d.y * (rhi.y - o.y)) +
         fmaxf(d.z * (rlo.z - o.z), d.z * (rhi.z - o.z));
}

// true when the first b reflections of a chain were all on static faces
__device__ inline bool static_chain(const uint32_t *fc, uint32_t b, uint32_t fs) {
  bool ok = true;
#pragma unroll
  for (uint32_t k = 0; k < EMRT_MAX_DEPTH; k++)
    if (k < b && fc[k] >= fs) ok = false;
  return ok;
}

// Closest-hit traversal of one bounce for every ray (persistent threads: each
// warp takes FETCH rays at a time from a global cursor).  BATCH: rays of many
// scenes, each ray's scene read from the table; otherwise the single scene in
// L.g.  Per ray: nearest hit over the static triangles and the vehicle
// boxes, reception-sphere detections on the traced segment (appended as
// candidates), and the specular continuation (appended to the next buffer).
// TABLE: static-hit cache form (single scene): the static hit of a segment
// whose chain is still static comes from L.stab when its entry is current,
// and is stored there otherwise.
template <bool BATCH, int BLOCK, int FETCH, bool WIDE, bool TABLE = false>
__global__ void __launch_bounds__(BLOCK, 1280 / BLOCK) k_bounce(BounceLaunch L, const BatchScene *__restrict__ tab,
                                                  uint32_t n_scenes) {
  int stk[kStack];
  float stt[kStack];
  TravStats st;
  uint32_t segs = 0, reused = 0;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t n_items = (L.b == 0 && !TABLE) ? L.n_primary : *L.n_in;
  float3 rlo, rhi;
  if (!BATCH) rx_bounds(L.g.rxb, rlo, rhi);
  const uint32_t NO = EMRT_NO_FACE;
  for (;;) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(L.work, (uint32_t)FETCH);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= n_items) break;
    for (uint32_t sub = 0; sub < (uint32_t)FETCH; sub += 32) {
      uint32_t i = base + sub + lane;
      if (i >= n_items) break;
      segs++;
      float3 o, d;
      float Lacc;
      uint32_t tx, j, sc = 0;
      uint32_t fc[EMRT_MAX_DEPTH] = {NO, NO, NO, NO};
      if (L.b == 0 && !TABLE) {
        uint32_t local = i, count = L.count;
        const float4 *dirs = L.dirs;
        if (BATCH) {  // scene of a primary item: last scene whose range starts <= i
          uint32_t lo = 0, hi = n_scenes;
          while (hi - lo > 1) {
            uint32_t mid = (lo + hi) >> 1;
            if (tab[mid].prim_begin <= i) lo = mid;
            else hi = mid;
          }
          sc = lo;
          local = i - tab[sc].prim_begin;
          count = tab[sc].count;
          dirs = tab[sc].dirs;
        }
        tx = local / count;
        uint32_t k = local - tx * count;
        float4 dj = dirs[k];
        d = f3(dj);
        j = __float_as_uint(dj.w);
        o = f3((BATCH ? tab[sc].g : L.g).tx_pos[tx]);
        Lacc = 0.f;
      } else {
        Ray R = L.rin[L.order ? L.order[i] : i];
        o = f3(R.o_L);
        Lacc = R.o_L.w;
        d = f3(R.d_id);
        uint32_t id = __float_as_uint(R.d_id.w);
        if (BATCH) {
          sc = id >> 26;
          tx = (id >> 22) & 15u;
          j = id & 0x3fffffu;
        } else {
          tx = id >> L.jbits;
          j = id & ((1u << L.jbits) - 1u);  // TABLE: direction-table position
        }
        fc[0] = R.faces.x; fc[1] = R.faces.y; fc[2] = R.faces.z; fc[3] = R.faces.w;
      }
      const GeomView &g = BATCH ? tab[sc].g : L.g;
      const float kappa = BATCH ? tab[sc].kappa : L.kappa;
      const int K = BATCH ? (int)tab[sc].K : L.K;
      if (BATCH) rx_bounds(g.rxb, rlo, rhi);
      uint32_t prev = L.b > 0 ? fc[L.b - 1] : NO;
      RayQ q;
      ray_setup(q, o, d);
      float tbest = FLT_MAX;
      uint32_t face = NO;
      bool have = false;
      uint32_t slot = 0, ep = 0;
      const bool keep = TABLE && static_chain(fc, (uint32_t)L.b, g.n_static_faces);
      if (keep) {
        slot = (uint32_t)L.b * L.n_slots + tx * L.count + j;
        ep = L.tx_epoch[tx];
        const uint4 e = L.stab[slot];
        if (e.z == ep) {
          tbest = __uint_as_float(e.x);
          face = e.y;
          have = true;
          reused++;
        }
      }
      if (!have) {
        trace_tris<false, WIDE>(g.stat, q, 0.f, tbest, face, prev, NO, stk, stt, st);
        if (keep) L.stab[slot] = make_uint4(__float_as_uint(tbest), face, ep, 0u);
      }
      uint32_t exv = (prev != NO && prev >= g.n_static_faces) ? (prev - g.n_static_faces) / 6u : NO;
      trace_boxes<false>(g.dyn, q, 0.f, tbest, face, g.n_static_faces, exv, NO, stk, stt, st);
      bool hit = face != NO;
      float t_end = hit ? tbest : escape_t(o, d, rlo, rhi);
      t_end = fmaxf(t_end, 0.f);
      float rmax = kappa * (Lacc + t_end) * 1.0001f + 1e-6f;
      const uint32_t b = (uint32_t)L.b;
      const uint32_t w0 = BATCH ? (sc << 8 | tx) : tx;
      query_rx(g.rxb, q, t_end, Lacc, kappa, rmax, stk, stt, st, [&](uint32_t rx) {
        uint32_t slot = warp_append(L.n_cand);
        if (slot < L.cand_cap) {
          const uint32_t jj = TABLE ? __float_as_uint(L.dirs[j].w) : j;
          uint4 *c = reinterpret_cast<uint4 *>(L.cand + 8ull * slot);
          c[0] = make_uint4(w0, rx, b, fc[0]);
          c[1] = make_uint4(fc[1], fc[2], fc[3], jj);
        }
      });
      if (hit && L.b < K) {
        float3 p, r;
        reflect_step(g, face, o, d, tbest, p, r);
        fc[L.b] = face;
        uint32_t slot = warp_append(L.n_out);
        Ray R;
        R.o_L = make_float4(p.x, p.y, p.z, Lacc + tbest);
        uint32_t id = BATCH ? (sc << 26 | tx << 22 | j) : (tx << L.jbits | j);
        R.d_id = make_float4(r.x, r.y, r.z, __uint_as_float(id));
        R.faces = make_uint4(fc[0], fc[1], fc[2], fc[3]);
        L.rout[slot] = R;
      }
    }
  }
  __syncwarp();
  add_u64(&L.ctr->segments[L.b], segs);
  add_u64(&L.ctr->node_visits, st.nodes);
  add_u64(&L.ctr->tri_tests, st.tris);
  add_u64(&L.ctr->dyn_node_visits, st.dnodes);
  add_u64(&L.ctr->box_tests, st.boxes);
  add_u64(&L.ctr->rx_node_visits, st.rnodes);
  add_u64(&L.ctr->rx_tests, st.rxs);
  if (TABLE) add_u64(&L.ctr->static_reused, reused);
  if (st.overflow) atomicOr(&L.ctr->err, ERR_STACK);
}

// Chain walker of the static-hit cache: one thread follows the whole specular
// chain of a primary ray (tx, direction-table position k) as long as its
// segments have current cache entries and its reflections stay on static
// faces: static hit from the cache, vehicle boxes and reception spheres of
// this frame, reflection.  The first segment it cannot finish that way (no
// current entry, or the chain reflected off a vehicle) goes to D.rays[b] for
// the per-bounce traversal, which continues the chain.  Segments, candidates
// and continuations are exactly those of k_bounce.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1280 / BLOCK) k_chain(BounceLaunch L, ChainBufs D) {
  int stk[kStack];
  float stt[kStack];
  TravStats st;
  uint32_t segs[EMRT_MAX_DEPTH + 1] = {0, 0, 0, 0, 0};
  uint32_t reused = 0, deferred = 0;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t n_items = L.n_primary;
  const uint32_t fs = L.g.n_static_faces;
  const uint32_t NO = EMRT_NO_FACE;
  float3 rlo, rhi;
  rx_bounds(L.g.rxb, rlo, rhi);
  for (;;) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(L.work, 32u);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= n_items) break;
    const uint32_t i = base + lane;
    if (i >= n_items) continue;
    const uint32_t tx = i / L.count;
    const uint32_t k = i - tx * L.count;
    const float4 dj = L.dirs[k];
    const uint32_t j = __float_as_uint(dj.w);
    const uint32_t ep = L.tx_epoch[tx];
    const uint32_t id = tx << L.jbits | k;
    float3 o = f3(L.g.tx_pos[tx]), d = f3(dj);
    float Lacc = 0.f;
    uint32_t f0 = NO, f1 = NO, f2 = NO, f3_ = NO;
    int defer_b = -1;
    for (int b = 0; b <= L.K; b++) {
      const uint4 e = L.stab[(uint32_t)b * L.n_slots + i];
      if (e.z != ep) {
        defer_b = b;
        break;
      }
      float tbest = __uint_as_float(e.x);
      uint32_t face = e.y;
      reused++;
      segs[b]++;
      RayQ q;
      ray_setup(q, o, d);
      // the face just left is static, so no vehicle is excluded
      trace_boxes<false>(L.g.dyn, q, 0.f, tbest, face, fs, NO, NO, stk, stt, st);
      const bool hit = face != NO;
      float t_end = hit ? tbest : escape_t(o, d, rlo, rhi);
      t_end = fmaxf(t_end, 0.f);
      const float rmax = L.kappa * (Lacc + t_end) * 1.0001f + 1e-6f;
      const uint32_t bb = (uint32_t)b;
      query_rx(L.g.rxb, q, t_end, Lacc, L.kappa, rmax, stk, stt, st, [&](uint32_t rx) {
        uint32_t slot = warp_append(L.n_cand);
        if (slot < L.cand_cap) {
          uint4 *c = reinterpret_cast<uint4 *>(L.cand + 8ull * slot);
          c[0] = make_uint4(tx, rx, bb, f0);
          c[1] = make_uint4(f1, f2, f3_, j);
        }
      });
      if (!hit || b == L.K) break;
      float3 p, r;
      reflect_step(L.g, face, o, d, tbest, p, r);
      f0 = b == 0 ? face : f0;
      f1 = b == 1 ? face : f1;
      f2 = b == 2 ? face : f2;
      f3_ = b == 3 ? face : f3_;
      Lacc = Lacc + tbest;
      o = p;
      d = r;
      if (face >= fs) {  // off a vehicle: the rest of the chain is not cached
        defer_b = b + 1;
        break;
      }
    }
    if (defer_b >= 0) {
      uint32_t slot = warp_append_keyed(L.ctr->n_ray, (uint32_t)defer_b);
      Ray R;
      R.o_L = make_float4(o.x, o.y, o.z, Lacc);
      R.d_id = make_float4(d.x, d.y, d.z, __uint_as_float(id));
      R.faces = make_uint4(f0, f1, f2, f3_);
      D.rays[defer_b][slot] = R;
      deferred++;
    }
  }
  __syncwarp();
  for (int b = 0; b <= EMRT_MAX_DEPTH; b++) add_u64(&L.ctr->segments[b], segs[b]);
  add_u64(&L.ctr->dyn_node_visits, st.dnodes);
  add_u64(&L.ctr->box_tests, st.boxes);
  add_u64(&L.ctr->rx_node_visits, st.rnodes);
  add_u64(&L.ctr->rx_tests, st.rxs);
  add_u64(&L.ctr->static_reused, reused);
  add_u64(&L.ctr->deferred, deferred);
  if (st.overflow) atomicOr(&L.ctr->err, ERR_STACK);
}

__global__ void k_tx_epoch(const float4 *pos, float4 *ref, uint32_t *epoch, uint32_t n) {
  uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float4 a = pos[t], r = ref[t];
  if (__float_as_uint(a.x) != __float_as_uint(r.x) || __float_as_uint(a.y) != __float_as_uint(r.y) ||
      __float_as_uint(a.z) != __float_as_uint(r.z)) {
    epoch[t] += 1u;
    ref[t] = a;
  }
}

// ----------------------------------------------------------------------------
// canonical key: tx | rx | depth | f0 | .. | f_{K-1}, most significant first
struct U128 { unsigned long long hi, lo; };
__device__ inline void push_bits(U128 &k, uint64_t v, int nb) {
  if (nb == 0) return;
  k.hi = (k.hi << nb) | (nb < 64 ? (k.lo >> (64 - nb)) : k.lo);
  k.lo = (nb < 64) ? ((k.lo << nb) | v) : v;
}

__global__ void k_path_keys(const uint32_t *rec, const uint32_t *n, uint32_t cap, KeyLayout kl,
                            KeyW<4> *keys, uint32_t *vals, uint32_t *n_eff) {
  uint32_t cnt = min(*n, cap);
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *n_eff = cnt;
  for (; i < cnt; i += gridDim.x * blockDim.x) {
    const uint4 *r = reinterpret_cast<const uint4 *>(rec + 8ull * i);
    uint4 a = r[0], b = r[1];
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
    keys[i] = kk;
    vals[i] = i;
  }
}

__device__ inline bool key_eq(const KeyW<4> &a, const KeyW<4> &b) {
  return a.w[0] == b.w[0] && a.w[1] == b.w[1] && a.w[2] == b.w[2] && a.w[3] == b.w[3];
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
    double4 p = g.face_plane[f];
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

template <bool BATCH>
__global__ void __launch_bounds__(kBounceBlock) k_accept(GeomView G, const BatchScene *__restrict__ tab,
                                                         uint32_t *rec, const uint32_t *n,
                                                         Counters *ctr) {
  int stk[kStack];
  float stt[kStack];
  TravStats st;
  uint32_t cnt = *n;
  unsigned long long occl = 0;
  const uint32_t NO = EMRT_NO_FACE;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
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
    D3 Q[EMRT_MAX_DEPTH + 2];
    if (ok) {
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
      // occlusion of the k+1 legs, endpoint faces excluded
      for (uint32_t q = 0; ok && q <= k; q++) {
        float3 A = make_float3((float)Q[q].x, (float)Q[q].y, (float)Q[q].z);
        float3 B = make_float3((float)Q[q + 1].x, (float)Q[q + 1].y, (float)Q[q + 1].z);
        uint32_t e0 = q >= 1 ? f[q - 1] : NO, e1 = q < k ? f[q] : NO;
        uint32_t v0 = (e0 != NO && e0 >= g.n_static_faces) ? (e0 - g.n_static_faces) / 6u : NO;
        uint32_t v1 = (e1 != NO && e1 >= g.n_static_faces) ? (e1 - g.n_static_faces) / 6u : NO;
        RayQ rq;
        ray_setup(rq, A, B - A);
        float tmax = 1.f;
        uint32_t hf = NO;
        occl++;
        TravStats s2;
        if (trace_tris<true>(g.stat, rq, 0.f, tmax, hf, e0, e1, stk, stt, s2)) ok = false;
        tmax = 1.f;
        if (ok && trace_boxes<true>(g.dyn, rq, 0.f, tmax, hf, g.n_static_faces, v0, v1, stk, stt, s2))
          ok = false;
        st.overflow |= s2.overflow;
      }
    }
    uint32_t flags = (ok ? EMRT_PATH_VALID : 0u) | (marg ? EMRT_PATH_MARGINAL : 0u);
    a.z = (a.z & 15u) | flags;
    r[0] = a;
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

__device__ inline uint32_t spread7(uint32_t v) {  // 7 bits -> every third bit
  uint32_t x = v & 0x7fu;
  x = (x | (x << 8)) & 0x0000f00fu;
  x = (x | (x << 4)) & 0x000c30c3u;
  x = (x | (x << 2)) & 0x00249249u;
  return x;
}

__global__ void k_ray_keys(const Ray *r, const uint32_t *n, const float4 *bb, KeyW<1> *keys,
                           uint32_t *vals, bool batched) {
  uint32_t cnt = *n;
  float4 lo = bb[0], hi = bb[1];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    float4 o = r[i].o_L, d = r[i].d_id;
    uint32_t c[3];
    float q[3] = {(o.x - lo.x) / (hi.x - lo.x), (o.y - lo.y) / (hi.y - lo.y), (o.z - lo.z) / (hi.z - lo.z)};
    for (int k = 0; k < 3; k++) c[k] = (uint32_t)(fminf(fmaxf(q[k], 0.f), 1.f) * 127.f);
    uint32_t m = spread7(c[0]) << 2 | spread7(c[1]) << 1 | spread7(c[2]);
    uint32_t oc = oct_code(make_float3(d.x, d.y, d.z));
    keys[i].w[0] = batched ? ((__float_as_uint(d.w) >> 26) << 26 | (m >> 1) << 6 | oc >> 26)
                           : (m << 11 | oc >> 21);
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

void launch_chain(const BounceLaunch &L, const ChainBufs &D, int grid, cudaStream_t s) {
  emrt::note_launch(), k_chain<kBounceBlock><<<grid, kBounceBlock, 0, s>>>(L, D);
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
  int grid;
};
Variant g_variants[] = {
    {"block64_fetch32", 64, k_bounce<true, 64, 32, false>, 0},
    {"block128_fetch32", 128, k_bounce<true, 128, 32, false>, 0},
    {"block256_fetch32", 256, k_bounce<true, 256, 32, false>, 0},
    {"block128_fetch128", 128, k_bounce<true, 128, 128, false>, 0},
    {"block256_fetch64", 256, k_bounce<true, 256, 64, false>, 0},
    {"block64_fetch128", 64, k_bounce<true, 64, 128, false>, 0},
    {"block128_fetch32_bvh4", 128, k_bounce<true, 128, 32, true>, 0},
    {"block64_fetch32_bvh4", 64, k_bounce<true, 64, 32, true>, 0},
};
constexpr int kNumVariants = sizeof(g_variants) / sizeof(g_variants[0]);
}  // namespace

int n_bounce_variants() { return kNumVariants; }
const char *bounce_variant_name(int v) { return g_variants[v].name; }
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
                           cudaStream_t s) {
  GeomView none{};
  emrt::note_launch(), k_accept<true><<<kPrimGrid * 4, kBounceBlock, 0, s>>>(none, tab, rec, n, ctr);
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
  if (L.stab)
    emrt::note_launch(), k_bounce<false, kBounceBlock, 32, false, true><<<grid, kBounceBlock, 0, s>>>(L, nullptr, 1);
  else if (wide)
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
                   cudaStream_t s) {
  emrt::note_launch(), k_accept<false><<<kPrimGrid * 4, kBounceBlock, 0, s>>>(g, nullptr, rec, n, ctr);
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
