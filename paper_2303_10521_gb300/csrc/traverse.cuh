// Stack traversal of the binary LBVH: closest hit and any hit over triangles
// (watertight test) and vehicle boxes (slab test with entry face), and the
// reception-sphere query over the receiver points.
//
// Node and primitive loads are 16-byte vector loads through the read-only
// path (ld.global.nc).  The ray/triangle test is the watertight algorithm of
// Woop, Benthin and Wald (JCGT 2013), restated from the publication: shear
// the triangle into ray space, evaluate the three 2D edge functions without
// FMA contraction (so both triangles sharing an edge see the same value) and
// re-evaluate them in double precision when one of them is exactly zero.
#pragma once
#include "common.cuh"

namespace emrt {

constexpr int kStack = 64;
// traversal stack entry: node code and entry distance, one 8-byte access
struct __align__(8) StackSlot {
  int node;
  float t;
};
// hard bound on loop iterations per query (a safety net: a well-formed tree
// never comes close); exceeding it records a device error and stops
constexpr uint32_t kMaxIter = 1u << 22;

struct RayQ {
  float3 o, d, idir, ood;
  int kx, ky, kz;
  float Sx, Sy, Sz;
};

__device__ inline float sel3(float3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }
__device__ inline float4 ldg4(const float4 *p) { return __ldg(p); }

__device__ inline void ray_setup(RayQ &r, float3 o, float3 d) {
  r.o = o;
  r.d = d;
  const float tiny = 1e-30f;
  float3 dd = make_float3(fabsf(d.x) < tiny ? copysignf(tiny, d.x) : d.x,
                          fabsf(d.y) < tiny ? copysignf(tiny, d.y) : d.y,
                          fabsf(d.z) < tiny ? copysignf(tiny, d.z) : d.z);
  r.idir = make_float3(1.f / dd.x, 1.f / dd.y, 1.f / dd.z);
  r.ood = make_float3(o.x * r.idir.x, o.y * r.idir.y, o.z * r.idir.z);
  float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
  int kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
  int kx = kz == 2 ? 0 : kz + 1;
  int ky = kx == 2 ? 0 : kx + 1;
  float dz = sel3(d, kz);
  if (dz < 0.f) { int t = kx; kx = ky; ky = t; }
  r.kx = kx; r.ky = ky; r.kz = kz;
  r.Sz = 1.f / dz;
  r.Sx = sel3(d, kx) * r.Sz;
  r.Sy = sel3(d, ky) * r.Sz;
}

// slab test of one child box against [tmin, tmax]; conservative far bound
__device__ inline bool slab(const RayQ &r, float lx, float hx, float ly, float hy, float lz, float hz,
                            float tmin, float tmax, float &tnear) {
  float t0x = fmaf(lx, r.idir.x, -r.ood.x), t1x = fmaf(hx, r.idir.x, -r.ood.x);
  float t0y = fmaf(ly, r.idir.y, -r.ood.y), t1y = fmaf(hy, r.idir.y, -r.ood.y);
  float t0z = fmaf(lz, r.idir.z, -r.ood.z), t1z = fmaf(hz, r.idir.z, -r.ood.z);
  float tn = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fmaxf(fminf(t0z, t1z), tmin));
  float tf = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fminf(fmaxf(t0z, t1z), tmax));
  tnear = tn;
  return tn <= tf * 1.00000024f;
}

// Two FMAs in one packed f32x2 instruction (sm_100 and later); each lane is
// rounded exactly like fmaf, so results equal the scalar form bit for bit.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 pa, pb, pc, pd;\n\t"
      "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\tmov.b64 pc, {%6, %7};\n\t"
      "fma.rn.f32x2 pd, pa, pb, pc;\n\tmov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

// The ray's slab terms as lane pairs for ffma2, per axis (idir, idir) and
// the origin terms of the low and the high plane, (-ol, -oh): t = p idir - ol
// for the low planes, p idir - oh for the high ones.  ray_pairs(): ol = oh =
// o idir, slab() exactly; ray_pairs_lh() with ol = (o + e) idir and oh =
// (o - e) idir tests the box grown by e on every side.
struct RayPairs {
  float2 ix, iy, iz, ox, oy, oz;
};
__device__ inline RayPairs ray_pairs(const RayQ &r) {
  return RayPairs{make_float2(r.idir.x, r.idir.x), make_float2(r.idir.y, r.idir.y),
                  make_float2(r.idir.z, r.idir.z), make_float2(-r.ood.x, -r.ood.x),
                  make_float2(-r.ood.y, -r.ood.y), make_float2(-r.ood.z, -r.ood.z)};
}
__device__ inline RayPairs ray_pairs_lh(const float3 &idir, const float3 &ol, const float3 &oh) {
  return RayPairs{make_float2(idir.x, idir.x), make_float2(idir.y, idir.y),
                  make_float2(idir.z, idir.z), make_float2(-ol.x, -oh.x),
                  make_float2(-ol.y, -oh.y), make_float2(-ol.z, -oh.z)};
}

// slab() with the low and the high plane of each axis in one packed FMA
__device__ inline bool slab_p(const RayPairs &q, float lx, float hx, float ly, float hy, float lz,
                              float hz, float tmin, float tmax, float &tnear) {
  const float2 tx = ffma2(make_float2(lx, hx), q.ix, q.ox);
  const float2 ty = ffma2(make_float2(ly, hy), q.iy, q.oy);
  const float2 tz = ffma2(make_float2(lz, hz), q.iz, q.oz);
  float tn = fmaxf(fmaxf(fminf(tx.x, tx.y), fminf(ty.x, ty.y)), fmaxf(fminf(tz.x, tz.y), tmin));
  float tf = fminf(fminf(fmaxf(tx.x, tx.y), fmaxf(ty.x, ty.y)), fminf(fmaxf(tz.x, tz.y), tmax));
  tnear = tn;
  return tn <= tf * 1.00000024f;
}

// Watertight ray/triangle test; on a hit with tmin < t < tmax returns t.
__device__ inline bool tri_hit(const RayQ &r, float3 v0, float3 v1, float3 v2, float tmin,
                               float tmax, float &t) {
  float3 A = v0 - r.o, B = v1 - r.o, C = v2 - r.o;
  float Akz = sel3(A, r.kz), Bkz = sel3(B, r.kz), Ckz = sel3(C, r.kz);
  float Ax = __fsub_rn(sel3(A, r.kx), __fmul_rn(r.Sx, Akz));
  float Ay = __fsub_rn(sel3(A, r.ky), __fmul_rn(r.Sy, Akz));
  float Bx = __fsub_rn(sel3(B, r.kx), __fmul_rn(r.Sx, Bkz));
  float By = __fsub_rn(sel3(B, r.ky), __fmul_rn(r.Sy, Bkz));
  float Cx = __fsub_rn(sel3(C, r.kx), __fmul_rn(r.Sx, Ckz));
  float Cy = __fsub_rn(sel3(C, r.ky), __fmul_rn(r.Sy, Ckz));
  float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
  float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
  float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
  if (U == 0.f || V == 0.f || W == 0.f) {
    U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
    V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
    W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
  }
  if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return false;
  float det = U + V + W;
  if (det == 0.f) return false;
  float Az = r.Sz * Akz, Bz = r.Sz * Bkz, Cz = r.Sz * Ckz;
  float T = U * Az + V * Bz + W * Cz;
  float adet = fabsf(det);
  float aT = det < 0.f ? -T : T;
  if (aT <= tmin * adet || aT >= tmax * adet) return false;
  t = T / det;
  return t > tmin && t < tmax;
}

struct TravStats {
  uint32_t nodes = 0, tris = 0, dnodes = 0, boxes = 0, rnodes = 0, rxs = 0;
  bool overflow = false;
};
#define EMRT_ITER_GUARD(st)            \
  if (++iter > kMaxIter) {             \
    st.overflow = true;                \
    return hit;                        \
  }

// Triangles first .. first + cnt - 1 of `prims`: watertight tests, exclusion
// of faces ex0/ex1, closest-hit tie to the lower face ID.  Returns true when
// tmax/face changed.
template <bool ANY>
__device__ inline bool tri_range(const float4 *prims, uint32_t first, uint32_t cnt,
                                 const RayQ &r, float tmin, float &tmax, uint32_t &face,
                                 uint32_t ex0, uint32_t ex1, TravStats &st) {
  bool changed = false;
  for (uint32_t q = 0; q < cnt; q++) {
    const float4 *tp = prims + 3ull * (first + q);
    float4 a = ldg4(tp), bb = ldg4(tp + 1), c = ldg4(tp + 2);
    st.tris++;
    uint32_t f = __float_as_uint(a.w);
    float t;
    // closest hit: widen the bound slightly so that an exact tie can go to
    // the lower face ID; any hit: strictly inside (tmin, tmax)
    if (f != ex0 && f != ex1 &&
        tri_hit(r, f3(a), f3(bb), f3(c), tmin, ANY ? tmax : tmax * 1.0000001f, t)) {
      if (t < tmax || (!ANY && t == tmax && f < face)) {
        tmax = t;
        face = f;
        changed = true;
        if (ANY) return true;
      }
    }
  }
  return changed;
}

// One triangle leaf (1-4 triangles, see BVHView::leaf_bits).
template <bool ANY>
__device__ inline bool leaf_tri(const BVHView &b, uint32_t code, const RayQ &r, float tmin,
                                float &tmax, uint32_t &face, uint32_t ex0, uint32_t ex1,
                                TravStats &st) {
  const uint32_t g0 = b.leaf_bits ? code >> 2 : code;
  const uint32_t cnt = b.leaf_bits ? (code & 3u) + 1u : 1u;
  return tri_range<ANY>(b.prims, g0, cnt, r, tmin, tmax, face, ex0, ex1, st);
}

// Compressed 8-wide traversal (node layout in BVHView::nodes8).  Per node:
// one 80-byte fetch, the 8 quantised child boxes decoded and slab-tested in
// straight-line code, the hits turned into a mask in visiting order (bit k =
// slot k ^ o, o the ray's sign pattern: roughly near to far, no sort).  The
// stack holds node groups -- first child, inner-slot mask and the children
// still to visit -- so one entry serves up to 7 siblings.  A lane descends
// until it holds leaf children to test (then the warp's leaf tests run
// together), tests them nearest slot first, and continues.
__device__ inline uint32_t wide_kmask(uint32_t v, uint32_t oct) {
  // bit s of each byte -> bit s ^ oct
  if (oct & 1u) v = ((v & 0x5555u) << 1) | ((v >> 1) & 0x5555u);
  if (oct & 2u) v = ((v & 0x3333u) << 2) | ((v >> 2) & 0x3333u);
  if (oct & 4u) v = ((v & 0x0f0fu) << 4) | ((v >> 4) & 0x0f0fu);
  return v;
}

template <bool ANY>
__device__ inline bool trace_tris8(const BVHView &b, const RayQ &r, float tmin, float &tmax,
                                   uint32_t &face, uint32_t ex0, uint32_t ex1, StackSlot *stk,
                                   TravStats &st) {
  const bool nx = r.idir.x < 0.f, ny = r.idir.y < 0.f, nz = r.idir.z < 0.f;
  const uint32_t oct = (nx ? 1u : 0u) | (ny ? 2u : 0u) | (nz ? 4u : 0u);
  bool hit = false;
  int sp = 0;
  uint32_t iter = 0;
  uint32_t gb = 0, gi = 0, gk = 0;               // inner group: first child, mask, to visit
  uint32_t lb = 0, lk = 0, lm0 = 0, lm1 = 0;      // leaf group: first tri, to test, meta
  uint32_t node = 0;                              // the root is visited first
  for (;;) {
    while (lk == 0) {
      if (++iter > kMaxIter) {
        st.overflow = true;
        return hit;
      }
      if (iter > 1) {
        if (gk == 0) {
          if (sp == 0) return hit;
          sp--;
          gb = (uint32_t)stk[sp].node & 0xffffffu;
          gi = (uint32_t)stk[sp].node >> 24;
          gk = __float_as_uint(stk[sp].t);
        }
        const uint32_t s = (uint32_t)(__ffs(gk) - 1) ^ oct;
        gk &= gk - 1u;
        node = gb + __popc(gi & ((1u << s) - 1u));
        if (gk) {
          if (sp < kStack) {
            stk[sp] = StackSlot{(int)(gb | gi << 24), __uint_as_float(gk)};
            sp++;
          } else {
            st.overflow = true;
          }
        }
      }
      const uint4 *np = b.nodes8 + 5ull * node;
      const uint4 h0 = __ldg(np), h1 = __ldg(np + 1), qx = __ldg(np + 2), qy = __ldg(np + 3),
                  qz = __ldg(np + 4);
      st.nodes++;
      // t of grid coordinate q along an axis: (2^23 + q) * ax + cx, the
      // 2^23 offset coming from the byte-to-float conversion
      const float ax = __uint_as_float((h0.w & 0xffu) << 23) * r.idir.x;
      const float ay = __uint_as_float(((h0.w >> 8) & 0xffu) << 23) * r.idir.y;
      const float az = __uint_as_float(((h0.w >> 16) & 0xffu) << 23) * r.idir.z;
      const float cx = fmaf(-8388608.f, ax, fmaf(__uint_as_float(h0.x), r.idir.x, -r.ood.x));
      const float cy = fmaf(-8388608.f, ay, fmaf(__uint_as_float(h0.y), r.idir.y, -r.ood.y));
      const float cz = fmaf(-8388608.f, az, fmaf(__uint_as_float(h0.z), r.idir.z, -r.ood.z));
      // near and far planes by the direction's sign
      const uint32_t nx0 = nx ? qx.z : qx.x, nx1 = nx ? qx.w : qx.y;
      const uint32_t fx0 = nx ? qx.x : qx.z, fx1 = nx ? qx.y : qx.w;
      const uint32_t ny0 = ny ? qy.z : qy.x, ny1 = ny ? qy.w : qy.y;
      const uint32_t fy0 = ny ? qy.x : qy.z, fy1 = ny ? qy.y : qy.w;
      const uint32_t nz0 = nz ? qz.z : qz.x, nz1 = nz ? qz.w : qz.y;
      const uint32_t fz0 = nz ? qz.x : qz.z, fz1 = nz ? qz.y : qz.w;
      // near and far plane of an axis in one packed FMA
      const float2 ax2 = make_float2(ax, ax), ay2 = make_float2(ay, ay), az2 = make_float2(az, az);
      const float2 cx2 = make_float2(cx, cx), cy2 = make_float2(cy, cy), cz2 = make_float2(cz, cz);
      uint32_t hits = 0;
#pragma unroll
      for (int sl = 0; sl < 8; sl++) {
        const uint32_t sel = 0x7440u | (uint32_t)(sl & 3);
        const float2 tx = ffma2(
            make_float2(__uint_as_float(__byte_perm(sl < 4 ? nx0 : nx1, 0x4B000000u, sel)),
                        __uint_as_float(__byte_perm(sl < 4 ? fx0 : fx1, 0x4B000000u, sel))),
            ax2, cx2);
        const float2 ty = ffma2(
            make_float2(__uint_as_float(__byte_perm(sl < 4 ? ny0 : ny1, 0x4B000000u, sel)),
                        __uint_as_float(__byte_perm(sl < 4 ? fy0 : fy1, 0x4B000000u, sel))),
            ay2, cy2);
        const float2 tz = ffma2(
            make_float2(__uint_as_float(__byte_perm(sl < 4 ? nz0 : nz1, 0x4B000000u, sel)),
                        __uint_as_float(__byte_perm(sl < 4 ? fz0 : fz1, 0x4B000000u, sel))),
            az2, cz2);
        const float tn = fmaxf(fmaxf(tx.x, ty.x), fmaxf(tz.x, tmin));
        const float tf = fminf(fminf(tx.y, ty.y), fminf(tz.y, tmax));
        if (tn <= tf * 1.00000024f) hits |= 1u << sl;
      }
      const uint32_t imask = h0.w >> 24, lmask = h1.x >> 24;
      const uint32_t k = wide_kmask((hits & imask) | (hits & lmask) << 8, oct);
      gb = h1.x & 0xffffffu;
      gi = imask;
      gk = k & 0xffu;
      lk = k >> 8;
      lb = h1.y;
      lm0 = h1.z;
      lm1 = h1.w;
    }
    // leaf children of the last node, nearest slot first
    while (lk) {
      const uint32_t s = (uint32_t)(__ffs(lk) - 1) ^ oct;
      lk &= lk - 1u;
      const uint32_t meta = __byte_perm(lm0, lm1, s) & 0xffu;
      if (tri_range<ANY>(b.prims8, lb + (meta & 31u), ((meta >> 5) & 3u) + 1u, r, tmin, tmax,
                         face, ex0, ex1, st)) {
        hit = true;
        if (ANY) return true;
      }
    }
  }
}

// Closest hit (ANY = false) or any hit (ANY = true) over the triangle BVH with
// t in (tmin, tmax).  Triangles of faces ex0/ex1 are skipped.  On a hit
// tmax and face are updated.  Ties in t go to the lower face ID.
// WIDE: use the compressed 8-wide tree when the BVH has one.
template <bool ANY, bool WIDE = false>
__device__ inline bool trace_tris(const BVHView &b, const RayQ &r, float tmin, float &tmax,
                                  uint32_t &face, uint32_t ex0, uint32_t ex1, StackSlot *stk,
                                  TravStats &st) {
  if (b.n_prims == 0) return false;
  if (WIDE && b.nodes8 && b.n_prims >= 2)
    return trace_tris8<ANY>(b, r, tmin, tmax, face, ex0, ex1, stk, st);
  bool hit = false;
  int sp = 0;
  int node = b.root;
  // node visits bound the loop (every leaf visit follows a visit or a pop of
  // an entry a visit pushed): a well-formed tree never comes close
  const uint32_t lim = st.nodes > 0xffffffffu - kMaxIter ? 0xffffffffu : st.nodes + kMaxIter;
  // a popped subtree is skipped only when its entry lies beyond the bound
  // with the slab test's own slack (closest hit), so that pruning on pop and
  // on visit agree and exact ties in t can still reach the lower face ID
  const float pop_slack = ANY ? 1.f : 1.00000024f;
  const RayPairs rp = ray_pairs(r);
  for (;;) {
    // descend through inner nodes until this lane reaches a leaf, so that
    // the lanes of a warp test their leaves together
    while (node >= 0) {
      if (st.nodes >= lim) {
        st.overflow = true;
        return hit;
      }
      const float4 *np = b.nodes + 4ll * node;
      float4 n0 = ldg4(np), n1 = ldg4(np + 1), n2 = ldg4(np + 2), n3 = ldg4(np + 3);
      st.nodes++;
      float tn0, tn1;
      bool h0 = slab_p(rp, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, tmin, tmax, tn0);
      bool h1 = slab_p(rp, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, tmin, tmax, tn1);
      int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
      if (h0 && h1) {
        int nearc = c0, farc = c1;
        float tfar = tn1;
        if (tn1 < tn0) { nearc = c1; farc = c0; tfar = tn0; }
        if (sp < kStack) { stk[sp] = StackSlot{farc, tfar}; sp++; }
        else st.overflow = true;
        node = nearc;
        continue;
      }
      if (h0) { node = c0; continue; }
      if (h1) { node = c1; continue; }
      // pop the next subtree that can still hold a closer hit
      for (;;) {
        if (sp == 0) return hit;
        sp--;
        if (stk[sp].t <= tmax * pop_slack) break;
      }
      node = stk[sp].node;
    }
    if (leaf_tri<ANY>(b, (uint32_t)(~node), r, tmin, tmax, face, ex0, ex1, st)) {
      hit = true;
      if (ANY) return true;
    }
    for (;;) {
      if (sp == 0) return hit;
      sp--;
      if (stk[sp].t <= tmax * pop_slack) break;
    }
    node = stk[sp].node;
  }
}

// One vehicle-box leaf: entry hit with t in (tmin, tmax) unless the box is
// excluded (vehicle exv0 or exv1); face = fs + 6 v + entry face.  Returns
// true when tmax/face changed.
__device__ inline bool leaf_box(const BVHView &b, uint32_t g, const RayQ &r, float tmin,
                                float &tmax, uint32_t &face, uint32_t fs, uint32_t exv0,
                                uint32_t exv1) {
  float4 lo = ldg4(b.prims + 2ull * g), hi = ldg4(b.prims + 2ull * g + 1);
  uint32_t v = __float_as_uint(lo.w);
  if (v == exv0 || v == exv1) return false;
  float tx0 = (lo.x - r.o.x) * r.idir.x, tx1 = (hi.x - r.o.x) * r.idir.x;
  float ty0 = (lo.y - r.o.y) * r.idir.y, ty1 = (hi.y - r.o.y) * r.idir.y;
  float tz0 = (lo.z - r.o.z) * r.idir.z, tz1 = (hi.z - r.o.z) * r.idir.z;
  float nx = fminf(tx0, tx1), ny = fminf(ty0, ty1), nz = fminf(tz0, tz1);
  float tn = fmaxf(nx, fmaxf(ny, nz));
  float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fmaxf(tz0, tz1));
  if (!(tn <= tf && tn > tmin && tn < tmax)) return false;
  int axis = (tn == nx) ? 0 : ((tn == ny) ? 1 : 2);
  float dax = axis == 0 ? r.d.x : (axis == 1 ? r.d.y : r.d.z);
  tmax = tn;
  face = fs + 6u * v + 2u * axis + (dax > 0.f ? 0u : 1u);
  return true;
}

// Vehicle boxes: closest (or any) entry hit with t in (tmin, tmax).  Box v is
// skipped when exv0 or exv1 equals v.  face = F_s + 6 v + entry face.
template <bool ANY>
__device__ inline bool trace_boxes(const BVHView &b, const RayQ &r, float tmin, float &tmax,
                                   uint32_t &face, uint32_t fs, uint32_t exv0, uint32_t exv1,
                                   StackSlot *stk, TravStats &st) {
  if (b.n_prims == 0) return false;
  const RayPairs rp = ray_pairs(r);
  bool hit = false;
  int sp = 0;
  int node = b.root;
  uint32_t iter = 0;
  for (;;) {
    EMRT_ITER_GUARD(st)
    if (node >= 0) {
      const float4 *np = b.nodes + 4ll * node;
      float4 n0 = ldg4(np), n1 = ldg4(np + 1), n2 = ldg4(np + 2), n3 = ldg4(np + 3);
      st.dnodes++;
      float tn0, tn1;
      bool h0 = slab_p(rp, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, tmin, tmax, tn0);
      bool h1 = slab_p(rp, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, tmin, tmax, tn1);
      int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
      if (h0 && h1) {
        int nearc = c0, farc = c1;
        float tfar = tn1;
        if (tn1 < tn0) { nearc = c1; farc = c0; tfar = tn0; }
        if (sp < kStack) { stk[sp] = StackSlot{farc, tfar}; sp++; }
        else st.overflow = true;
        node = nearc;
        continue;
      }
      if (h0) { node = c0; continue; }
      if (h1) { node = c1; continue; }
    } else {
      st.boxes++;
      if (leaf_box(b, (uint32_t)(~node), r, tmin, tmax, face, fs, exv0, exv1)) {
        hit = true;
        if (ANY) return true;
      }
    }
    for (;;) {
      if (sp == 0) return hit;
      sp--;
      if (stk[sp].t <= tmax) break;
    }
    node = stk[sp].node;
  }
}

// Exact reception-sphere test of receiver position p against the segment
// o + s d, s in [0, t_end], unfolded length L at o.
__device__ inline bool rx_hit(float4 p, const RayQ &r, float t_end, float L, float kappa) {
  float3 w = f3(p) - r.o;
  float s = fminf(fmaxf(dot3(w, r.d), 0.f), t_end);
  float3 q = w - r.d * s;
  float rad = kappa * (L + s);
  return dot3(q, q) <= rad * rad;
}

// Vehicle boxes and receivers in one traversal of the merged per-frame tree
// (prims 0..n_veh-1 are vehicle boxes, the others receiver points, stored as
// empty boxes with their receiver index + n_veh in lo.w).  Vehicles: closest
// entry hit with t in (0, tmax), exactly as trace_boxes<false> (vehicle exv
// skipped; tmax and face updated).  Receivers: collected into rx_buf (at most
// RXB; more sets rx_over) when their box grown by rmax is entered within tq,
// the bound of the segment end known before the call (the static hit or the
// escape distance), which shrinks with every vehicle hit; rmax must bound
// the reception radius at tq.  The caller tests the collected receivers
// exactly (rx_hit) with the final segment end.  Boxes are grown by rmax for
// the vehicles too, which only widens their pruning.
template <int RXB>
__device__ inline void trace_veh_rx(const BVHView &b, const RayQ &r, float &tmax, uint32_t &face,
                                    uint32_t fs, uint32_t n_veh, uint32_t exv, float tq,
                                    float rmax, uint32_t *rx_buf, int &n_rx, bool &rx_over,
                                    StackSlot *stk, TravStats &st) {
  if (b.n_prims == 0) return;
  const float3 ol = make_float3(r.ood.x + rmax * r.idir.x, r.ood.y + rmax * r.idir.y,
                                r.ood.z + rmax * r.idir.z);
  const float3 oh = make_float3(r.ood.x - rmax * r.idir.x, r.ood.y - rmax * r.idir.y,
                                r.ood.z - rmax * r.idir.z);
  const RayPairs rp = ray_pairs_lh(r.idir, ol, oh);
  int sp = 0;
  int node = b.root;
  float tcur = 0.f;  // entry distance of the node being visited
  uint32_t iter = 0;
  for (;;) {
    if (++iter > kMaxIter) {
      st.overflow = true;
      return;
    }
    if (node >= 0) {
      const float4 *np = b.nodes + 4ll * node;
      float4 n0 = ldg4(np), n1 = ldg4(np + 1), n2 = ldg4(np + 2), n3 = ldg4(np + 3);
      st.dnodes++;
      float tn0, tn1;
      bool h0 = slab_p(rp, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, 0.f, tmax, tn0);
      bool h1 = slab_p(rp, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, 0.f, tmax, tn1);
      int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
      if (h0 && h1) {
        int nearc = c0, farc = c1;
        float tnear = tn0, tfar = tn1;
        if (tn1 < tn0) { nearc = c1; farc = c0; tnear = tn1; tfar = tn0; }
        if (sp < kStack) { stk[sp] = StackSlot{farc, tfar}; sp++; }
        else st.overflow = true;
        node = nearc;
        tcur = tnear;
        continue;
      }
      if (h0) { node = c0; tcur = tn0; continue; }
      if (h1) { node = c1; tcur = tn1; continue; }
    } else {
      const uint32_t gi = (uint32_t)(~node);
      const uint32_t s = __float_as_uint(ldg4(b.prims + 2ull * gi).w);
      if (s < n_veh) {
        st.boxes++;
        if (leaf_box(b, gi, r, 0.f, tmax, face, fs, exv, EMRT_NO_FACE)) tq = fminf(tq, tmax);
      } else if (tcur <= tq) {
        st.rxs++;
        if (n_rx < RXB) rx_buf[n_rx++] = s - n_veh;
        else rx_over = true;
      }
    }
    for (;;) {
      if (sp == 0) return;
      sp--;
      if (stk[sp].t <= tmax) break;
    }
    node = stk[sp].node;
    tcur = stk[sp].t;
  }
}

// Reception spheres: for every receiver p whose distance to the segment
// o + s d, s in [0, t_end], is <= kappa (L + s) at the segment point nearest
// to p, calls emit(receiver id).  rmax bounds kappa (L + t_end).
template <typename F>
__device__ inline void query_rx(const BVHView &b, const RayQ &r, float t_end, float L, float kappa,
                                float rmax, StackSlot *stk, TravStats &st, F &&emit) {
  if (b.n_prims == 0) return;
  int sp = 0;
  int node = b.root;
  uint32_t iter = 0;
  const bool hit = false;
  for (;;) {
    if (++iter > kMaxIter) {
      st.overflow = true;
      return;
    }
    (void)hit;
    if (node >= 0) {
      const float4 *np = b.nodes + 4ll * node;
      float4 n0 = ldg4(np), n1 = ldg4(np + 1), n2 = ldg4(np + 2), n3 = ldg4(np + 3);
      st.rnodes++;
      float tn0, tn1;
      bool h0 = slab(r, n0.x - rmax, n0.y + rmax, n0.z - rmax, n0.w + rmax, n2.x - rmax,
                     n2.y + rmax, 0.f, t_end, tn0);
      bool h1 = slab(r, n1.x - rmax, n1.y + rmax, n1.z - rmax, n1.w + rmax, n2.z - rmax,
                     n2.w + rmax, 0.f, t_end, tn1);
      int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
      if (h0 && h1) {
        if (sp < kStack) { stk[sp] = StackSlot{c1, 0.f}; sp++; }
        else st.overflow = true;
        node = c0;
        continue;
      }
      if (h0) { node = c0; continue; }
      if (h1) { node = c1; continue; }
    } else {
      float4 p = ldg4(b.prims + (uint32_t)(~node));
      st.rxs++;
      if (rx_hit(p, r, t_end, L, kappa)) emit(__float_as_uint(p.w));
    }
    if (sp == 0) return;
    node = stk[--sp].node;
  }
}

}  // namespace emrt
