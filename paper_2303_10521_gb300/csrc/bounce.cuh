// Closest-hit traversal kernel of one discovery bounce (k_bounce) with the
// device helpers it shares with the static-hit cache walker (chain.cuh).
// Included by trace.cu only, inside its anonymous namespace.
#pragma once

__device__ inline float3 face_normal_f(const GeomView &g, uint32_t f) {
  if (f < g.n_static_faces) {
    double4_32a p = g.face_plane[f];
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

// Receivers buffered per segment by the merged query (in local memory).  A
// segment that meets more takes the receiver-tree query instead, a second
// traversal with grown boxes; with 4 those were the cache walker's slowest
// chunks at low ray densities (large reception spheres): 64 took the city's
// N/10 rediscovery walk from 0.66-0.73 to 0.52-0.60 ms, 128 and 256 gained
// nothing more, and the full-density traces did not change.
constexpr int kRxBuf = 64;

// Vehicle boxes and reception spheres of one segment after its static
// closest hit (tbest, face): one traversal of the merged vehicle + receiver
// tree when the scene has one (collected receivers are tested exactly with
// the final segment end; more than kRxBuf falls back to the receiver tree),
// the two separate queries otherwise.  Same hits and detections either way.
// Updates tbest/face; returns whether the segment hit something.
template <typename F>
__device__ inline bool veh_and_rx(const GeomView &g, const RayQ &q, float3 o, float3 d,
                                  float3 rlo, float3 rhi, float Lacc, float kappa, uint32_t exv,
                                  float &tbest, uint32_t &face, StackSlot *stk,
                                  TravStats &st, F &&emit) {
  const uint32_t NO = EMRT_NO_FACE;
  if (g.mix.n_prims) {
    const float tq = fmaxf(face != NO ? tbest : escape_t(o, d, rlo, rhi), 0.f);
    const float rq = kappa * (Lacc + tq) * 1.0001f + 1e-6f;
    uint32_t rxb[kRxBuf];
    int nrx = 0;
    bool over = false;
    trace_veh_rx<kRxBuf>(g.mix, q, tbest, face, g.n_static_faces, g.n_veh, exv, tq, rq, rxb, nrx,
                         over, stk, st);
    const bool hit = face != NO;
    const float t_end = fmaxf(hit ? tbest : escape_t(o, d, rlo, rhi), 0.f);
    if (over) {
      const float rmax = kappa * (Lacc + t_end) * 1.0001f + 1e-6f;
      query_rx(g.rxb, q, t_end, Lacc, kappa, rmax, stk, st, emit);
    } else {
      for (int k = 0; k < nrx; k++)
        if (rx_hit(g.rx_pos[rxb[k]], q, t_end, Lacc, kappa)) emit(rxb[k]);
    }
    return hit;
  }
  trace_boxes<false>(g.dyn, q, 0.f, tbest, face, g.n_static_faces, exv, NO, stk, st);
  const bool hit = face != NO;
  const float t_end = fmaxf(hit ? tbest : escape_t(o, d, rlo, rhi), 0.f);
  const float rmax = kappa * (Lacc + t_end) * 1.0001f + 1e-6f;
  query_rx(g.rxb, q, t_end, Lacc, kappa, rmax, stk, st, emit);
  return hit;
}

// Closest-hit traversal of one bounce for every ray (persistent threads: each
// warp takes FETCH rays at a time from a global cursor).  BATCH: rays of many
// scenes, each ray's scene read from the table; otherwise the single scene in
// L.g.  Per ray: nearest hit over the static triangles and the vehicle
// boxes, reception-sphere detections on the traced segment (appended as
// candidates), and the specular continuation (appended to the next buffer).
template <bool BATCH, int BLOCK, int FETCH, bool WIDE>
__global__ void __launch_bounds__(BLOCK, 1280 / BLOCK) k_bounce(BounceLaunch L, const BatchScene *__restrict__ tab,
                                                  uint32_t n_scenes) {
  StackSlot stk[kStack];
  TravStats st;
  uint32_t segs = 0;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t n_items = L.b == 0 ? L.n_primary : *L.n_in;
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
      if (L.b == 0) {
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
          j = id & ((1u << L.jbits) - 1u);
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
      trace_tris<false, WIDE>(g.stat, q, 0.f, tbest, face, prev, NO, stk, st);
      uint32_t exv = (prev != NO && prev >= g.n_static_faces) ? (prev - g.n_static_faces) / 6u : NO;
      const uint32_t b = (uint32_t)L.b;
      const uint32_t w0 = BATCH ? (sc << 8 | tx) : tx;
      const bool hit = veh_and_rx(g, q, o, d, rlo, rhi, Lacc, kappa, exv, tbest, face, stk, st,
                                  [&](uint32_t rx) {
        uint32_t slot = warp_append(L.n_cand);
        if (slot < L.cand_cap) {
          uint4 *c = reinterpret_cast<uint4 *>(L.cand + 8ull * slot);
          c[0] = make_uint4(w0, rx, b, fc[0]);
          c[1] = make_uint4(fc[1], fc[2], fc[3], j);
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
        if (!BATCH && L.okeys) {
          L.okeys[slot].w[0] = ray_key(p, r, L.bbox[0], L.bbox[1]);
          L.ovals[slot] = slot;
        }
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
  if (st.overflow) atomicOr(&L.ctr->err, ERR_STACK);
}
