// Depth-first discovery kernels: the static-hit cache walker (k_chain), the
// walk without the cache (k_walk), and the epoch kernel of the cache's
// transmitter positions.  Included by trace.cu only, after bounce.cuh, inside
// its anonymous namespace.
#pragma once

// One chain from its first unfinished segment to its end, in scene g (kappa:
// reception radius factor, K: reflections).  CACHE (single scene): static
// hit from the cache L.stab while the chain is still static and its entry
// (tx, item = tx * count + direction-table position) is current, the full
// static traversal otherwise (stored when the chain is static); without: the
// full static traversal.  Then the vehicle boxes and reception spheres of
// this frame, and the reflection.  R holds the origin, L travelled, direction
// and faces met; the segment index b of its first segment is the number of
// faces met.  Candidates carry w0 in word 0 and jj (the ray index) in word 7.
// Segments, candidates and cache entries are exactly those of k_bounce.
template <bool CACHE, bool WIDE = false>
__device__ __forceinline__ void carry_chain(const BounceLaunch &L, const GeomView &g, float kappa,
                                            int K, uint32_t w0, uint32_t tx, uint32_t item,
                                            uint32_t jj, const Ray &R, float3 rlo, float3 rhi,
                                            StackSlot *stk, TravStats &st,
                                            uint32_t (&segs)[EMRT_MAX_DEPTH + 1],
                                            uint32_t &reused) {
  const uint32_t fs = g.n_static_faces;
  const uint32_t NO = EMRT_NO_FACE;
  float3 o = f3(R.o_L), d = f3(R.d_id);
  float Lacc = R.o_L.w;
  uint32_t f0 = R.faces.x, f1 = R.faces.y, f2 = R.faces.z, f3_ = R.faces.w;
  uint32_t b = (f0 != NO) + (f1 != NO) + (f2 != NO) + (f3_ != NO);
  for (;;) {
    const uint32_t prev = b == 0 ? NO : b == 1 ? f0 : b == 2 ? f1 : b == 3 ? f2 : f3_;
    RayQ q;
    ray_setup(q, o, d);
    float tbest = FLT_MAX;
    uint32_t face = NO;
    bool have = false;
    uint32_t slot = 0, ep = 0;
    const bool keep = CACHE && (b < 1 || f0 < fs) && (b < 2 || f1 < fs) && (b < 3 || f2 < fs) &&
                      (b < 4 || f3_ < fs);
    if (keep) {
      slot = b * L.n_slots + item;
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
      trace_tris<false, WIDE>(g.stat, q, 0.f, tbest, face, prev, NO, stk, st);
      if (keep) L.stab[slot] = make_uint4(__float_as_uint(tbest), face, ep, 0u);
    }
    const uint32_t exv = (prev != NO && prev >= fs) ? (prev - fs) / 6u : NO;
    const uint32_t bb = b;
    const bool hit = veh_and_rx(g, q, o, d, rlo, rhi, Lacc, kappa, exv, tbest, face, stk, st,
                                [&](uint32_t rx) {
      uint32_t s = warp_append(L.n_cand);
      if (s < L.cand_cap) {
        uint4 *c = reinterpret_cast<uint4 *>(L.cand + 8ull * s);
        c[0] = make_uint4(w0, rx, bb, f0);
        c[1] = make_uint4(f1, f2, f3_, jj);
      }
    });
#pragma unroll
    for (uint32_t k = 0; k <= EMRT_MAX_DEPTH; k++)
      if (k == b) segs[k]++;
    if (!hit || (int)b >= K) break;
    float3 p, r;
    reflect_step(g, face, o, d, tbest, p, r);
    f0 = b == 0 ? face : f0;
    f1 = b == 1 ? face : f1;
    f2 = b == 2 ? face : f2;
    f3_ = b == 3 ? face : f3_;
    Lacc = Lacc + tbest;
    o = p;
    d = r;
    b++;
  }
}

// A chain of the walker's queue: R.d_id.w holds tx << L.jbits | position in
// the direction table.
__device__ __forceinline__ void carry_queued(const BounceLaunch &L, const Ray &R, float3 rlo,
                                             float3 rhi, StackSlot *stk, TravStats &st,
                                             uint32_t (&segs)[EMRT_MAX_DEPTH + 1],
                                             uint32_t &reused) {
  const uint32_t id = __float_as_uint(R.d_id.w);
  const uint32_t tx = id >> L.jbits, pos = id & ((1u << L.jbits) - 1u);
  carry_chain<true>(L, L.g, L.kappa, L.K, tx, tx, tx * L.count + pos,
                    __float_as_uint(L.dirs[pos].w), R, rlo, rhi, stk, st, segs, reused);
}

// Chain walker of the static-hit cache.  Walk tasks: one thread follows the
// whole specular chain of a primary ray (tx, direction-table position k) as
// long as its segments have current cache entries and its reflections stay on
// static faces: static hit from the cache, vehicle boxes and reception
// spheres of this frame, reflection.  A chain it cannot finish that way (no
// current entry, or a reflection off a vehicle) goes to the warp's own queue
// (kChainQueue entries of D.q, written and read by this warp alone); as soon
// as it holds 32 chains the warp carries them to their ends together
// (carry_chain), so that the costly deferred segments run while the walk
// still fills the GPU, 32 to a warp, rather than in a sparse launch of their
// own.  The queue's last chains are carried when the walk is handed out.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1280 / BLOCK) k_chain(BounceLaunch L, ChainBufs D) {
  StackSlot stk[kStack];
  TravStats st;
  uint32_t segs[EMRT_MAX_DEPTH + 1] = {0, 0, 0, 0, 0};
  uint32_t reused = 0, deferred = 0;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t n_items = L.n_primary;
  const uint32_t fs = L.g.n_static_faces;
  const uint32_t NO = EMRT_NO_FACE;
  Ray *wq = D.q + (size_t)(blockIdx.x * (BLOCK / 32) + (threadIdx.x >> 5)) * kChainQueue;
  uint32_t qn = 0;  // chains in the warp's queue (warp-uniform)
  float3 rlo, rhi;
  rx_bounds(L.g.rxb, rlo, rhi);
  for (;;) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(L.work, 32u);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= n_items) break;
    const uint32_t i = base + lane;
    bool defer = false;
    float3 o, d;
    float Lacc = 0.f;
    uint32_t id = 0, f0 = NO, f1 = NO, f2 = NO, f3_ = NO;
    if (i < n_items) {
      const uint32_t tx = i / L.count;
      const uint32_t k = i - tx * L.count;
      const float4 dj = L.dirs[k];
      const uint32_t j = __float_as_uint(dj.w);
      const uint32_t ep = L.tx_epoch[tx];
      id = tx << L.jbits | k;
      o = f3(L.g.tx_pos[tx]);
      d = f3(dj);
      for (int b = 0; b <= L.K; b++) {
        const uint4 e = L.stab[(uint32_t)b * L.n_slots + i];
        if (e.z != ep) {
          defer = true;
          break;
        }
        float tbest = __uint_as_float(e.x);
        uint32_t face = e.y;
        reused++;
        segs[b]++;
        RayQ q;
        ray_setup(q, o, d);
        // the face just left is static, so no vehicle is excluded
        const uint32_t bb = (uint32_t)b;
        const bool hit = veh_and_rx(L.g, q, o, d, rlo, rhi, Lacc, L.kappa, NO, tbest, face, stk,
                                    st, [&](uint32_t rx) {
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
          defer = true;
          break;
        }
      }
    }
    const uint32_t m = __ballot_sync(0xffffffffu, defer);
    if (defer) {
      Ray *q = wq + qn + __popc(m & lanemask_lt());
      q->o_L = make_float4(o.x, o.y, o.z, Lacc);
      q->d_id = make_float4(d.x, d.y, d.z, __uint_as_float(id));
      q->faces = make_uint4(f0, f1, f2, f3_);
      deferred++;
    }
    qn += __popc(m);
    if (qn >= 32u) {  // carry the queue's last 32 chains
      __syncwarp();
      const Ray R = wq[qn - 32u + lane];
      __syncwarp();
      qn -= 32u;
      carry_queued(L, R, rlo, rhi, stk, st, segs, reused);
    }
  }
  __syncwarp();
  if (lane < qn) carry_queued(L, wq[lane], rlo, rhi, stk, st, segs, reused);
  __syncwarp();
  for (int b = 0; b <= EMRT_MAX_DEPTH; b++) add_u64(&L.ctr->segments[b], segs[b]);
  add_u64(&L.ctr->node_visits, st.nodes);
  add_u64(&L.ctr->tri_tests, st.tris);
  add_u64(&L.ctr->dyn_node_visits, st.dnodes);
  add_u64(&L.ctr->box_tests, st.boxes);
  add_u64(&L.ctr->rx_node_visits, st.rnodes);
  add_u64(&L.ctr->rx_tests, st.rxs);
  add_u64(&L.ctr->static_reused, reused);
  add_u64(&L.ctr->deferred, deferred);
  if (st.overflow) atomicOr(&L.ctr->err, ERR_STACK);
}

// Depth-first discovery without the cache: a warp takes 32 neighbouring
// primary rays (tx, direction-table positions k .. k + 31, neighbouring
// directions) from the global cursor L.work and carries each chain to its end
// (carry_chain), the 32 chains in lockstep.  Measured on the city against the
// breadth-first form (k_bounce per bounce with the coherence sort): the
// chains of neighbouring directions stay coherent through their bounces, and
// there are no ray buffers, sorts or per-bounce launches.  Handing a lane
// whose chain ended a new primary ray at once was slower: it mixes depths in
// a warp.  BATCH: primary items of many scenes (table tab, each item's scene
// the last whose range starts at or before it; candidates carry
// scene << 8 | tx); otherwise the single scene in L.g.  Segments and
// candidates are exactly those of k_bounce.  WIDE: closest hits through the
// compressed 8-wide tree of the static geometry (same hits).
template <int BLOCK, bool BATCH, bool WIDE = false>
__global__ void __launch_bounds__(BLOCK, (WIDE ? 1024 : 1280) / BLOCK) k_walk(BounceLaunch L,
                                                             const BatchScene *__restrict__ tab,
                                                             uint32_t n_scenes) {
  StackSlot stk[kStack];
  TravStats st;
  uint32_t segs[EMRT_MAX_DEPTH + 1] = {0, 0, 0, 0, 0};
  uint32_t unused = 0;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t n_items = L.n_primary;
  const uint32_t NO = EMRT_NO_FACE;
  float3 rlo, rhi;
  if (!BATCH) rx_bounds(L.g.rxb, rlo, rhi);
  for (;;) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(L.work, 32u);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= n_items) break;
    const uint32_t i = base + lane;
    if (i < n_items) {
      uint32_t sc = 0, local = i, count = L.count;
      const float4 *dirs = L.dirs;
      if (BATCH) {
        uint32_t lo = 0, hi = n_scenes;
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (tab[mid].prim_begin <= i) lo = mid;
          else hi = mid;
        }
        sc = lo;
        local = i - tab[sc].prim_begin;
        count = tab[sc].count;
        dirs = tab[sc].dirs;
      }
      const GeomView &g = BATCH ? tab[sc].g : L.g;
      if (BATCH) rx_bounds(g.rxb, rlo, rhi);
      const uint32_t tx = local / count;
      const uint32_t k = local - tx * count;
      const float4 p = g.tx_pos[tx], dj = dirs[k];
      Ray R;
      R.o_L = make_float4(p.x, p.y, p.z, 0.f);
      R.d_id = dj;
      R.faces = make_uint4(NO, NO, NO, NO);
      carry_chain<false, WIDE>(L, g, BATCH ? tab[sc].kappa : L.kappa, BATCH ? (int)tab[sc].K : L.K,
                         BATCH ? (sc << 8 | tx) : tx, tx, local, __float_as_uint(dj.w), R, rlo,
                         rhi, stk, st, segs, unused);
    }
    __syncwarp();
  }
  for (int k = 0; k <= EMRT_MAX_DEPTH; k++) add_u64(&L.ctr->segments[k], segs[k]);
  add_u64(&L.ctr->node_visits, st.nodes);
  add_u64(&L.ctr->tri_tests, st.tris);
  add_u64(&L.ctr->dyn_node_visits, st.dnodes);
  add_u64(&L.ctr->box_tests, st.boxes);
  add_u64(&L.ctr->rx_node_visits, st.rnodes);
  add_u64(&L.ctr->rx_tests, st.rxs);
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
