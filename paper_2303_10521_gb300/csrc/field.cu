// Per-path complex field (Sec. III-C), per-(tx, rx) statistics (Table III,
// Sec. V-D) and the adjoint of the coherent sums with respect to material
// permittivity, conductivity and transmitter position.
//
// One generic routine computes the field of a path for a scalar type T.  With
// T = double it is the forward kernel; with T = Dual<N> (value plus N
// tangents) the same arithmetic carries derivatives with respect to the
// transmitter coordinates and the (eps_r, sigma) of every bounce, so the
// adjoint recomputes reflection points instead of storing Jacobians.  Path
// length and phase are accumulated in FP64 (L / lambda formed in double).
#include "field.cuh"

namespace emrt {

namespace {

constexpr double kC = 299792458.0;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// scalar abstraction
template <int N>
struct Dual {
  double v;
  double d[N];
  __device__ Dual() {}
  __device__ Dual(double x) : v(x) {
#pragma unroll
    for (int i = 0; i < N; i++) d[i] = 0.0;
  }
};

__device__ inline double val(double x) { return x; }
template <int N> __device__ inline double val(const Dual<N> &x) { return x.v; }

template <int N> __device__ inline Dual<N> operator+(const Dual<N> &a, const Dual<N> &b) {
  Dual<N> r; r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N> __device__ inline Dual<N> operator-(const Dual<N> &a, const Dual<N> &b) {
  Dual<N> r; r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N> __device__ inline Dual<N> operator-(const Dual<N> &a) {
  Dual<N> r; r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = -a.d[i];
  return r;
}
template <int N> __device__ inline Dual<N> operator*(const Dual<N> &a, const Dual<N> &b) {
  Dual<N> r; r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N> __device__ inline Dual<N> operator/(const Dual<N> &a, const Dual<N> &b) {
  Dual<N> r; r.v = a.v / b.v;
  double ib = 1.0 / b.v;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <int N> __device__ inline Dual<N> operator+(const Dual<N> &a, double b) { return a + Dual<N>(b); }
template <int N> __device__ inline Dual<N> operator-(const Dual<N> &a, double b) { return a - Dual<N>(b); }
template <int N> __device__ inline Dual<N> operator-(double a, const Dual<N> &b) { return Dual<N>(a) - b; }
template <int N> __device__ inline Dual<N> operator*(const Dual<N> &a, double b) {
  Dual<N> r; r.v = a.v * b;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = a.d[i] * b;
  return r;
}
template <int N> __device__ inline Dual<N> operator*(double b, const Dual<N> &a) { return a * b; }
template <int N> __device__ inline Dual<N> operator/(const Dual<N> &a, double b) { return a * (1.0 / b); }
template <int N> __device__ inline Dual<N> operator/(double a, const Dual<N> &b) { return Dual<N>(a) / b; }

__device__ inline double tsqrt(double x) { return sqrt(x); }
template <int N> __device__ inline Dual<N> tsqrt(const Dual<N> &a) {
  Dual<N> r; r.v = sqrt(a.v);
  double h = r.v > 0.0 ? 0.5 / r.v : 0.0;
#pragma unroll
  for (int i = 0; i < N; i++) r.d[i] = a.d[i] * h;
  return r;
}
__device__ inline double tabs(double x) { return fabs(x); }
template <int N> __device__ inline Dual<N> tabs(const Dual<N> &a) { return a.v < 0.0 ? -a : a; }
__device__ inline double tfrac(double x) { return x - floor(x); }
template <int N> __device__ inline Dual<N> tfrac(const Dual<N> &a) {
  Dual<N> r = a; r.v = a.v - floor(a.v); return r;
}
__device__ inline void tsincos(double x, double &s, double &c) { sincos(x, &s, &c); }
template <int N> __device__ inline void tsincos(const Dual<N> &x, Dual<N> &s, Dual<N> &c) {
  double sv, cv;
  sincos(x.v, &sv, &cv);
  s.v = sv; c.v = cv;
#pragma unroll
  for (int i = 0; i < N; i++) { s.d[i] = x.d[i] * cv; c.d[i] = -x.d[i] * sv; }
}

template <typename T> struct V3 { T x, y, z; };
template <typename T> __device__ inline V3<T> mk3(T x, T y, T z) { V3<T> r; r.x = x; r.y = y; r.z = z; return r; }
template <typename T> __device__ inline V3<T> operator+(const V3<T> &a, const V3<T> &b) { return mk3<T>(a.x + b.x, a.y + b.y, a.z + b.z); }
template <typename T> __device__ inline V3<T> operator-(const V3<T> &a, const V3<T> &b) { return mk3<T>(a.x - b.x, a.y - b.y, a.z - b.z); }
template <typename T, typename S> __device__ inline V3<T> scale(const V3<T> &a, const S &s) { return mk3<T>(a.x * s, a.y * s, a.z * s); }
template <typename T> __device__ inline T dot(const V3<T> &a, const V3<T> &b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T> __device__ inline V3<T> cross(const V3<T> &a, const V3<T> &b) {
  return mk3<T>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
template <typename T> __device__ inline V3<T> lift(double x, double y, double z) { return mk3<T>(T(x), T(y), T(z)); }

template <typename T> struct Cx { T re, im; };
template <typename T> __device__ inline Cx<T> cx(T r, T i) { Cx<T> c; c.re = r; c.im = i; return c; }
template <typename T> __device__ inline Cx<T> operator+(const Cx<T> &a, const Cx<T> &b) { return cx<T>(a.re + b.re, a.im + b.im); }
template <typename T> __device__ inline Cx<T> operator-(const Cx<T> &a, const Cx<T> &b) { return cx<T>(a.re - b.re, a.im - b.im); }
template <typename T> __device__ inline Cx<T> operator*(const Cx<T> &a, const Cx<T> &b) {
  return cx<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T> __device__ inline Cx<T> cscale(const Cx<T> &a, const T &s) { return cx<T>(a.re * s, a.im * s); }
template <typename T> __device__ inline Cx<T> operator/(const Cx<T> &a, const Cx<T> &b) {
  T den = b.re * b.re + b.im * b.im;
  return cx<T>((a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den);
}
// principal square root
template <typename T> __device__ inline Cx<T> csqrt_p(const Cx<T> &z) {
  T r = tsqrt(z.re * z.re + z.im * z.im);
  if (val(r) == 0.0) return cx<T>(T(0.0), T(0.0));
  if (val(z.re) >= 0.0) {
    T t = tsqrt((r + z.re) * 0.5);
    return cx<T>(t, z.im / (t * 2.0));
  }
  T t = tsqrt((r - z.re) * 0.5);
  if (val(z.im) >= 0.0) return cx<T>(z.im / (t * 2.0), t);
  return cx<T>(-(z.im) / (t * 2.0), -t);
}

template <typename T> struct CV3 { Cx<T> x, y, z; };
template <typename T> __device__ inline Cx<T> cdot(const CV3<T> &a, const V3<T> &b) {
  return cx<T>(a.x.re * b.x + a.y.re * b.y + a.z.re * b.z, a.x.im * b.x + a.y.im * b.y + a.z.im * b.z);
}

template <typename T> __device__ inline V3<T> unitv(const V3<T> &a) {
  T n = tsqrt(dot(a, a));
  return scale(a, T(1.0) / n);
}
// vertical transverse polarisation of the ideal omnidirectional antenna
template <typename T> __device__ inline V3<T> polar(const V3<T> &k) {
  V3<T> p = mk3<T>(T(0.0) - k.z * k.x, T(0.0) - k.z * k.y, T(1.0) - k.z * k.z);
  T n = tsqrt(dot(p, p));
  if (val(n) < 1e-12) return lift<T>(1.0, 0.0, 0.0);
  return scale(p, T(1.0) / n);
}

// ---------------------------------------------------------------------------
struct PathGeom {
  uint32_t k, f[EMRT_MAX_DEPTH];
  double n[EMRT_MAX_DEPTH][3];
  double d[EMRT_MAX_DEPTH];
  uint32_t mat[EMRT_MAX_DEPTH];
  float3 vel[EMRT_MAX_DEPTH];
};

// indices of a record within the scene (records written by the library
// always are; records supplied by a caller are checked before any load)
__device__ inline bool record_ok(const GeomView &g, const uint32_t *r) {
  uint32_t k = r[2] & 15u, nf = g.n_static_faces + 6u * g.n_veh;
  if (r[0] >= g.n_tx || r[1] >= g.n_rx || k > EMRT_MAX_DEPTH) return false;
  for (uint32_t q = 0; q < k; q++)
    if (r[3 + q] >= nf) return false;
  return true;
}

__device__ inline void load_geom(const GeomView &g, const uint32_t *rec, PathGeom &P) {
  uint4 a = reinterpret_cast<const uint4 *>(rec)[0], b = reinterpret_cast<const uint4 *>(rec)[1];
  P.k = min(a.z & 15u, (uint32_t)EMRT_MAX_DEPTH);
  uint32_t f[4] = {a.w, b.x, b.y, b.z};
  for (uint32_t q = 0; q < P.k; q++) {
    P.f[q] = f[q];
    if (f[q] < g.n_static_faces) {
      double4_32a p = g.face_plane[f[q]];
      P.n[q][0] = p.x; P.n[q][1] = p.y; P.n[q][2] = p.z; P.d[q] = p.w;
      P.mat[q] = g.face_info[f[q]].z;
      P.vel[q] = make_float3(0.f, 0.f, 0.f);
    } else {
      uint32_t v = (f[q] - g.n_static_faces) / 6u, j = (f[q] - g.n_static_faces) % 6u;
      int ax = j >> 1;
      bool neg = (j & 1u) == 0;
      float4 lo = g.veh_lo[v], hi = g.veh_hi[v];
      double s = neg ? -1.0 : 1.0;
      P.n[q][0] = ax == 0 ? s : 0.0; P.n[q][1] = ax == 1 ? s : 0.0; P.n[q][2] = ax == 2 ? s : 0.0;
      double c = ax == 0 ? (neg ? lo.x : hi.x) : (ax == 1 ? (neg ? lo.y : hi.y) : (neg ? lo.z : hi.z));
      P.d[q] = s * c;
      P.mat[q] = g.veh_mat;
      P.vel[q] = f3(g.veh_vel[v]);
    }
  }
}

// Geometry of one path (frequency-independent): image points, reflection
// points, the unfolded length L and the unit direction kh[q] of every leg.
// tx: transmitter position (seeded with tangents by the caller).
template <typename T>
__device__ inline void path_geometry(const PathGeom &P, V3<T> tx, V3<double> rx, T &Lout,
                                     V3<T> *kh) {
  const uint32_t k = P.k;
  V3<T> I[EMRT_MAX_DEPTH + 1], Q[EMRT_MAX_DEPTH + 2];
  I[0] = tx;
  for (uint32_t q = 0; q < k; q++) {
    V3<T> n = lift<T>(P.n[q][0], P.n[q][1], P.n[q][2]);
    T s = (dot(n, I[q]) - P.d[q]) * 2.0;
    I[q + 1] = I[q] - scale(n, s);
  }
  Q[0] = tx;
  Q[k + 1] = lift<T>(rx.x, rx.y, rx.z);
  for (int q = (int)k; q >= 1; q--) {
    V3<T> n = lift<T>(P.n[q - 1][0], P.n[q - 1][1], P.n[q - 1][2]);
    V3<T> D = Q[q + 1] - I[q];
    T t = (T(P.d[q - 1]) - dot(n, I[q])) / dot(n, D);
    Q[q] = I[q] + scale(D, t);
  }
  T L(0.0);
  for (uint32_t q = 0; q <= k; q++) {
    V3<T> D = Q[q + 1] - Q[q];
    T l = tsqrt(dot(D, D));
    L = L + l;
    kh[q] = scale(D, T(1.0) / l);
  }
  Lout = L;
}

// Field of a path of geometry (kh, L) at one frequency: polarisation
// transport through the Fresnel reflections, spreading and phase.
// epsr/sig: per-bounce material parameters.
template <typename T>
__device__ inline void path_transport(const PathGeom &P, const V3<T> *kh, T L, const T *epsr,
                                      const T *sig, const double *gam, bool const_gamma,
                                      double freq, Cx<T> &amp) {
  const uint32_t k = P.k;
  const double lam = kC / freq;
  V3<T> p0 = polar(kh[0]);
  CV3<T> E;
  E.x = cx<T>(p0.x, T(0.0)); E.y = cx<T>(p0.y, T(0.0)); E.z = cx<T>(p0.z, T(0.0));
  for (uint32_t q = 1; q <= k; q++) {
    V3<T> n = lift<T>(P.n[q - 1][0], P.n[q - 1][1], P.n[q - 1][2]);
    V3<T> kin = kh[q - 1], kout = kh[q];
    T cos_t = tabs(dot(kin, n));
    V3<T> sv = cross(kin, n);
    if (val(dot(sv, sv)) < 1e-24) {  // normal incidence: any s orthogonal to kin
      sv = cross(kin, lift<T>(1.0, 0.0, 0.0));
      if (val(dot(sv, sv)) < 1e-12) sv = cross(kin, lift<T>(0.0, 1.0, 0.0));
    }
    sv = unitv(sv);
    V3<T> pin = cross(sv, kin), pout = cross(sv, kout);
    Cx<T> gs, gp;
    if (const_gamma) {
      gs = cx<T>(T(-gam[q - 1]), T(0.0));
      gp = cx<T>(T(gam[q - 1]), T(0.0));
    } else {
      Cx<T> ec = cx<T>(epsr[q - 1], T(0.0) - sig[q - 1] * (1.0 / (2.0 * kPi * freq * kEps0)));
      T sin2 = T(1.0) - cos_t * cos_t;
      Cx<T> root = csqrt_p(cx<T>(ec.re - sin2, ec.im));
      Cx<T> ct = cx<T>(cos_t, T(0.0));
      gs = (ct - root) / (ct + root);
      Cx<T> ecct = cscale(ec, cos_t);
      gp = (ecct - root) / (ecct + root);
    }
    Cx<T> es = cdot(E, sv), ep = cdot(E, pin);
    Cx<T> a = gs * es, b = gp * ep;
    E.x = cscale(a, sv.x) + cscale(b, pout.x);
    E.y = cscale(a, sv.y) + cscale(b, pout.y);
    E.z = cscale(a, sv.z) + cscale(b, pout.z);
  }
  Cx<T> rcv = cdot(E, polar(kh[k]));
  T cyc = L * (1.0 / lam);
  T ph = tfrac(cyc) * (-2.0 * kPi);
  T sp, cp;
  tsincos(ph, sp, cp);
  T sc = T(lam / (4.0 * kPi)) / L;
  amp = cscale(rcv * cx<T>(cp, sp), sc);
}

// Field of one path at one frequency (geometry and transport).
template <typename T>
__device__ inline void path_field(const PathGeom &P, V3<T> tx, V3<double> rx, const T *epsr,
                                  const T *sig, const double *gam, bool const_gamma, double freq,
                                  Cx<T> &amp, T &Lout, V3<T> *kh) {
  path_geometry<T>(P, tx, rx, Lout, kh);
  path_transport<T>(P, kh, Lout, epsr, sig, gam, const_gamma, freq, amp);
}

// frequency q of a set (kernel parameters; no dynamic indexing)
__device__ inline void pick_freq(const FreqSet &fs, uint32_t q, double &freq, double *&out) {
  freq = fs.f[0];
  out = fs.path_out[0];
#pragma unroll
  for (uint32_t j = 1; j < kMaxFreq; j++)
    if (q == j) {
      freq = fs.f[j];
      out = fs.path_out[j];
    }
}

// Field of every path at the frequencies 2 blockIdx.y and 2 blockIdx.y + 1
// of fs: the path's geometry (image and reflection points, legs, Doppler
// rate) once, the transport at each of the two frequencies (the same
// arithmetic as for one frequency alone).
// A block takes kFieldBlock consecutive paths and hands them to its threads
// ordered by depth, so that a warp's paths mostly share their number of
// reflections: the per-bounce loops then run for the warp's own depth, not
// for the deepest path among 32 of every depth.  On GB300 each warp-wide FP64
// instruction holds the SM's FP64 units for many cycles whatever the number
// of active lanes, so lanes idled by shallower paths cost as much as busy
// ones.  Which thread computes a path does not change its result.
constexpr int kFieldBlock = 128;
__global__ void __launch_bounds__(kFieldBlock) k_field(GeomView g, MatView m, const uint32_t *rec,
                                                       const uint32_t *n, uint32_t cap,
                                                       FreqSet fs, Counters *ctr) {
  __shared__ uint32_t s_cnt[EMRT_MAX_DEPTH + 2];
  __shared__ uint32_t s_order[kFieldBlock];
  const uint32_t q0 = 2u * blockIdx.y;
  const bool two = q0 + 1u < fs.n;
  double freq0, freq1;
  double *out0, *out1;
  pick_freq(fs, q0, freq0, out0);
  pick_freq(fs, two ? q0 + 1u : q0, freq1, out1);
  const uint32_t cnt = min(*n, cap);
  for (uint32_t base = blockIdx.x * kFieldBlock; base < cnt; base += gridDim.x * kFieldBlock) {
    const uint32_t i = depth_ordered(rec, base, cnt, s_cnt, s_order);
    if (i >= cnt) continue;
    PathGeom P;
    const uint32_t *r = rec + 8ull * i;
    uint32_t tx = r[0], rx = r[1];
    if (!record_ok(g, r)) {  // malformed record: no field
      reinterpret_cast<double4_32a *>(out0)[i] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
      if (two) reinterpret_cast<double4_32a *>(out1)[i] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
      continue;
    }
    load_geom(g, r, P);
    double epsr[EMRT_MAX_DEPTH], sig[EMRT_MAX_DEPTH], gam[EMRT_MAX_DEPTH];
    for (uint32_t q = 0; q < P.k; q++) {
      uint32_t mm = min(P.mat[q], m.n_mat - 1);
      epsr[q] = m.eps_r[mm];
      sig[q] = m.sigma[mm];
      gam[q] = m.gamma ? m.gamma[mm] : 0.0;
    }
    float3 t3 = f3(g.tx_pos[tx]), r3 = f3(g.rx_pos[rx]);
    V3<double> txp = mk3<double>(t3.x, t3.y, t3.z), rxp = mk3<double>(r3.x, r3.y, r3.z);
    double L;
    V3<double> kh[EMRT_MAX_DEPTH + 1];
    path_geometry<double>(P, txp, rxp, L, kh);
    // Doppler: rate of change of the unfolded length (Eq. 3 generalised)
    float3 vt = f3(g.tx_vel[tx]), vr = f3(g.rx_vel[rx]);
    double dL = -(vt.x * kh[0].x + vt.y * kh[0].y + vt.z * kh[0].z) +
                (vr.x * kh[P.k].x + vr.y * kh[P.k].y + vr.z * kh[P.k].z);
    for (uint32_t q = 1; q <= P.k; q++) {
      float3 v = P.vel[q - 1];
      dL += v.x * (kh[q - 1].x - kh[q].x) + v.y * (kh[q - 1].y - kh[q].y) + v.z * (kh[q - 1].z - kh[q].z);
    }
    for (int f = 0; f < 2; f++) {
      if (f == 1 && !two) break;
      const double freq = f ? freq1 : freq0;
      Cx<double> a;
      path_transport<double>(P, kh, L, epsr, sig, gam, m.const_gamma != 0, freq, a);
      double4_32a o;
      o.x = a.re;
      o.y = a.im;
      o.z = L / kC;
      o.w = -(freq / kC) * dL;
      if (!isfinite(o.x) || !isfinite(o.y) || !isfinite(o.z) || !isfinite(o.w))
        atomicOr(&ctr->err, ERR_NONFINITE);
      reinterpret_cast<double4_32a *>(f ? out1 : out0)[i] = o;
    }
  }
}

// ---------------------------------------------------------------------------
// Per (tx, rx) statistics: the thread holding the first path of a run of
// equal (tx, rx) in the canonical order sums the run sequentially (fixed
// order, deterministic); pairs without paths keep the zeros written before.
__global__ void k_pair_seq(const uint32_t *rec, const uint32_t *n, uint32_t cap, uint32_t n_tx,
                           uint32_t n_rx, FreqSet fs) {
  const double *path_out = fs.path_out[0];
  double *pair_out = fs.pair_out[0];
#pragma unroll
  for (uint32_t q = 1; q < kMaxFreq; q++)
    if (blockIdx.y == q) {
      path_out = fs.path_out[q];
      pair_out = fs.pair_out[q];
    }
  uint32_t cnt = min(*n, cap);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    uint32_t tx = rec[8ull * i], rx = rec[8ull * i + 1];
    if (tx >= n_tx || rx >= n_rx) continue;
    if (i > 0 && rec[8ull * (i - 1)] == tx && rec[8ull * (i - 1) + 1] == rx) continue;
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    uint32_t e = i;
    for (; e < cnt && rec[8ull * e] == tx && rec[8ull * e + 1] == rx; e++) {
      double4_32a o = reinterpret_cast<const double4_32a *>(path_out)[e];
      double w = o.x * o.x + o.y * o.y;
      s[0] += o.x; s[1] += o.y; s[2] += w;
      s[3] += w * o.w; s[4] += w * o.w * o.w;
      s[5] += w * o.z; s[6] += w * o.z * o.z;
    }
    double *o = pair_out + 8ull * (tx * n_rx + rx);
    double pw = s[2];
    double fm = pw > 0 ? s[3] / pw : 0.0, tm = pw > 0 ? s[5] / pw : 0.0;
    double fv = pw > 0 ? s[4] / pw - fm * fm : 0.0, tv = pw > 0 ? s[6] / pw - tm * tm : 0.0;
    o[0] = s[0]; o[1] = s[1]; o[2] = pw;
    o[3] = fm; o[4] = sqrt(fmax(fv, 0.0));
    o[5] = tm; o[6] = sqrt(fmax(tv, 0.0));
    o[7] = (double)(e - i);
  }
}

__global__ void k_rx_power(uint32_t n_tx, uint32_t n_rx, double pt, FreqSet fs) {
  const double *pair_out = fs.pair_out[0];
  double *rx_out = fs.rx_out[0];
#pragma unroll
  for (uint32_t q = 1; q < kMaxFreq; q++)
    if (blockIdx.y == q) {
      pair_out = fs.pair_out[q];
      rx_out = fs.rx_out[q];
    }
  uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rx || !rx_out) return;
  double coh = 0.0, inc = 0.0;
  for (uint32_t t = 0; t < n_tx; t++) {
    const double *o = pair_out + 8ull * (t * n_rx + r);
    coh += o[0] * o[0] + o[1] * o[1];
    inc += o[2];
  }
  rx_out[2 * r] = pt * coh;
  rx_out[2 * r + 1] = pt * inc;
}

// ---------------------------------------------------------------------------
// adjoint: per path, tangents for tx (3) and (eps_r, sigma) of each bounce
constexpr int kTan = 3 + 2 * EMRT_MAX_DEPTH;
constexpr int kAdjBlock = 64;

__global__ void __launch_bounds__(kAdjBlock) k_field_tangents(GeomView g, MatView m,
                                                              const uint32_t *rec, const uint32_t *n,
                                                              uint32_t cap, double freq,
                                                              const double *dloss_dh, uint32_t n_rx,
                                                              double *contrib, Counters *ctr) {
  using D = Dual<kTan>;
  uint32_t cnt = min(*n, cap);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    PathGeom P;
    const uint32_t *r = rec + 8ull * i;
    uint32_t tx = r[0], rx = r[1];
    double *c = contrib + (size_t)kTan * i;
    if (!record_ok(g, r)) {
      for (int t = 0; t < kTan; t++) c[t] = 0.0;
      continue;
    }
    load_geom(g, r, P);
    D epsr[EMRT_MAX_DEPTH], sig[EMRT_MAX_DEPTH];
    double gam[EMRT_MAX_DEPTH];
    for (uint32_t q = 0; q < P.k; q++) {
      uint32_t mm = min(P.mat[q], m.n_mat - 1);
      epsr[q] = D(m.eps_r[mm]);
      epsr[q].d[3 + 2 * q] = 1.0;
      sig[q] = D(m.sigma[mm]);
      sig[q].d[4 + 2 * q] = 1.0;
      gam[q] = m.gamma ? m.gamma[mm] : 0.0;
    }
    float3 t3 = f3(g.tx_pos[tx]), r3 = f3(g.rx_pos[rx]);
    V3<D> txp = mk3<D>(D(t3.x), D(t3.y), D(t3.z));
    txp.x.d[0] = 1.0; txp.y.d[1] = 1.0; txp.z.d[2] = 1.0;
    V3<double> rxp = mk3<double>(r3.x, r3.y, r3.z);
    Cx<D> a;
    D L;
    V3<D> kh[EMRT_MAX_DEPTH + 1];
    path_field<D>(P, txp, rxp, epsr, sig, gam, m.const_gamma != 0, freq, a, L, kh);
    const double *gh = dloss_dh + 2ull * (tx * n_rx + rx);
    double gx = gh[0], gy = gh[1];
    bool finite = isfinite(a.re.v) && isfinite(a.im.v);
    for (int t = 0; t < kTan; t++) {
      c[t] = gx * a.re.d[t] + gy * a.im.d[t];
      finite = finite && isfinite(c[t]);
    }
    // a non-finite amplitude or tangent (e.g. NaN material parameters) is
    // reported as for the forward field
    if (!finite) atomicOr(&ctr->err, ERR_NONFINITE);
  }
}

// one block per gradient entry, fixed-order sum over paths
__global__ void k_grad_reduce(GeomView g, MatView m, const uint32_t *rec, const uint32_t *n,
                              uint32_t cap, const double *contrib, double *grad_eps,
                              double *grad_sigma, double *grad_tx) {
  __shared__ double sh[256];
  uint32_t cnt = min(*n, cap);
  uint32_t pid = blockIdx.x;  // [0, n_mat) eps, [n_mat, 2 n_mat) sigma, then tx*3+c
  double s = 0.0;
  for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    const uint32_t *r = rec + 8ull * i;
    const double *c = contrib + (size_t)kTan * i;
    if (pid < 2 * m.n_mat) {
      uint32_t mat = pid % m.n_mat;
      bool is_sig = pid >= m.n_mat;
      uint32_t k = min(r[2] & 15u, (uint32_t)EMRT_MAX_DEPTH);
      uint32_t f[4] = {r[3], r[4], r[5], r[6]};
      for (uint32_t q = 0; q < k; q++) {
        uint32_t fm = f[q] < g.n_static_faces ? g.face_info[f[q]].z : g.veh_mat;
        if (min(fm, m.n_mat - 1) == mat) s += c[3 + 2 * q + (is_sig ? 1 : 0)];
      }
    } else {
      uint32_t t = (pid - 2 * m.n_mat) / 3, comp = (pid - 2 * m.n_mat) % 3;
      if (r[0] == t) s += c[comp];
    }
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (pid < m.n_mat) grad_eps[pid] = sh[0];
    else if (pid < 2 * m.n_mat) grad_sigma[pid - m.n_mat] = sh[0];
    else grad_tx[pid - 2 * m.n_mat] = sh[0];
  }
}

// ---------------------------------------------------------------------------
// Channel statistics over time (Sec. III-B)
// Eq. 1 read as the normalised autocovariance of g = |h| over the frames:
// R(tau) = (mean_{t < F - tau} g(t) g(t + tau) - mu^2) / (mean g^2 - mu^2)
__global__ void k_correlation(const double *h, uint32_t F, uint32_t P, uint32_t L, double *R) {
  uint64_t id = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (uint64_t)P * (L + 1)) return;
  uint32_t p = (uint32_t)(id / (L + 1)), tau = (uint32_t)(id % (L + 1));
  double s1 = 0.0, s2 = 0.0;
  for (uint32_t t = 0; t < F; t++) {
    const double *z = h + 2ull * ((uint64_t)t * P + p);
    double g = sqrt(z[0] * z[0] + z[1] * z[1]);
    s1 += g;
    s2 += g * g;
  }
  double mu = s1 / F, var = s2 / F - mu * mu;
  double c = 0.0;
  uint32_t n = tau < F ? F - tau : 0;
  for (uint32_t t = 0; t < n; t++) {
    const double *a = h + 2ull * ((uint64_t)t * P + p);
    const double *b = h + 2ull * ((uint64_t)(t + tau) * P + p);
    c += sqrt(a[0] * a[0] + a[1] * a[1]) * sqrt(b[0] * b[0] + b[1] * b[1]);
  }
  double r = 0.0;
  if (n > 0 && var > 0.0) r = (c / n - mu * mu) / var;
  R[id] = r;
}

// Eq. 2 as printed: T_c = sqrt(1/R^4 - 1) / (2 pi f_D theta^2), f_D = f |v| / c
// the maximum Doppler shift of the receiver, theta the angle between its
// motion and the direction from the transmitter to the receiver
__device__ double coherence_time(const GeomView &g, uint32_t t, uint32_t r, double freq,
                                 double r_thr) {
  float3 a = f3(g.tx_pos[t]), b = f3(g.rx_pos[r]), v = f3(g.rx_vel[r]);
  double kx = (double)b.x - a.x, ky = (double)b.y - a.y, kz = (double)b.z - a.z;
  double kn = sqrt(kx * kx + ky * ky + kz * kz);
  double vn = sqrt((double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z);
  double out = INFINITY;
  if (kn > 0.0 && vn > 0.0) {
    double c = ((double)v.x * kx + (double)v.y * ky + (double)v.z * kz) / (kn * vn);
    double th = acos(fmin(1.0, fmax(-1.0, c)));
    double fd = freq * vn / kC;
    double den = 2.0 * kPi * fd * th * th;
    double num = sqrt(fmax(0.0, 1.0 / (r_thr * r_thr * r_thr * r_thr) - 1.0));
    if (den > 0.0) out = num / den;
  }
  return out;
}

__global__ void k_coherence(GeomView g, double freq, double r_thr, double *tc) {
  uint32_t id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= g.n_tx * g.n_rx) return;
  tc[id] = coherence_time(g, id / g.n_rx, id % g.n_rx, freq, r_thr);
}

// direct-path record of every (tx, rx) pair, pair i = tx * n_rx + rx
__global__ void k_los_records(uint32_t n_tx, uint32_t n_rx, uint32_t *rec) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_tx * n_rx) return;
  uint4 *c = reinterpret_cast<uint4 *>(rec + 8ull * i);
  c[0] = make_uint4(i / n_rx, i % n_rx, 0u, EMRT_NO_FACE);
  c[1] = make_uint4(EMRT_NO_FACE, EMRT_NO_FACE, EMRT_NO_FACE, 0u);
}

// Due rule of the per-receiver re-discovery schedule (see emrt.h).  los:
// the accepted direct-path records (w2 valid bit = line of sight).
__global__ void k_schedule(GeomView g, const uint32_t *los, float4 *state, uint8_t *los_ref,
                           double freq, double r_thr, double dt, float d_seg,
                           uint32_t max_interval, uint32_t *flag) {
  uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.n_rx) return;
  const float4 st = state[r];
  const float3 p = f3(g.rx_pos[r]);
  bool due = st.w < 0.f;
  double tc = INFINITY;
  for (uint32_t t = 0; t < g.n_tx; t++) {
    const uint32_t i = t * g.n_rx + r;
    const uint8_t now = (los[8ull * i + 2] & EMRT_PATH_VALID) ? 1 : 0;
    if (now != los_ref[i]) due = true;
    tc = fmin(tc, coherence_time(g, t, r, freq, r_thr));
  }
  const double dx = (double)p.x - st.x, dy = (double)p.y - st.y, dz = (double)p.z - st.z;
  if (dx * dx + dy * dy + dz * dz >= (double)d_seg * d_seg) due = true;
  double iv = dt > 0.0 ? floor(tc / dt) : INFINITY;  // frames within the coherence time
  uint32_t interval = iv >= (double)max_interval ? max_interval : (uint32_t)fmax(1.0, iv);
  const uint32_t frames = st.w < 0.f ? 0u : (uint32_t)st.w + 1u;
  if (frames >= interval) due = true;
  if (due) {
    state[r] = make_float4(p.x, p.y, p.z, 0.f);
    for (uint32_t t = 0; t < g.n_tx; t++) {
      const uint32_t i = t * g.n_rx + r;
      los_ref[i] = (los[8ull * i + 2] & EMRT_PATH_VALID) ? 1 : 0;
    }
  } else {
    state[r].w = (float)frames;
  }
  flag[r] = due ? 1u : 0u;
}

__global__ void k_compact_ids(const uint32_t *flag, const uint32_t *pos, uint32_t n,
                              uint32_t *ids) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flag[i]) ids[pos[i]] = i;
}

}  // namespace

void launch_correlation(const double *h, uint32_t n_frames, uint32_t n_pairs, uint32_t max_lag,
                        double *R, cudaStream_t s) {
  uint64_t n = (uint64_t)n_pairs * (max_lag + 1);
  emrt::note_launch(), k_correlation<<<ceil_div(n, 256), 256, 0, s>>>(h, n_frames, n_pairs, max_lag, R);
}

void launch_coherence(const GeomView &g, double freq, double r_thr, double *tc, cudaStream_t s) {
  emrt::note_launch(), k_coherence<<<ceil_div((uint64_t)g.n_tx * g.n_rx, 256), 256, 0, s>>>(g, freq, r_thr, tc);
}

void launch_los_records(uint32_t n_tx, uint32_t n_rx, uint32_t *rec, cudaStream_t s) {
  uint64_t n = (uint64_t)n_tx * n_rx;
  emrt::note_launch(), k_los_records<<<ceil_div(n, 256), 256, 0, s>>>(n_tx, n_rx, rec);
}

void launch_schedule(const GeomView &g, const uint32_t *los, float4 *state, uint8_t *los_ref,
                     double freq, double r_thr, double dt, float d_seg, uint32_t max_interval,
                     uint32_t *flag, cudaStream_t s) {
  emrt::note_launch(), k_schedule<<<ceil_div(g.n_rx, 128), 128, 0, s>>>(g, los, state, los_ref, freq, r_thr, dt, d_seg,
                                                        max_interval, flag);
}

void launch_compact_ids(const uint32_t *flag, const uint32_t *pos, uint32_t n, uint32_t *ids,
                        cudaStream_t s) {
  emrt::note_launch(), k_compact_ids<<<ceil_div(n, 256), 256, 0, s>>>(flag, pos, n, ids);
}

void launch_channel(const GeomView &g, MatView m, const uint32_t *rec, const uint32_t *n,
                    uint32_t cap, const FreqSet &fs, uint32_t n_tx, uint32_t n_rx,
                    double tx_power_w, Counters *ctr, cudaStream_t s) {
  // one grid row per pair of frequencies
  emrt::note_launch(), k_field<<<dim3(152 * 4, (fs.n + 1) / 2), kFieldBlock, 0, s>>>(g, m, rec, n, cap, fs, ctr);
  uint32_t np = n_tx * n_rx;
  for (uint32_t q = 0; q < fs.n; q++) cudaMemsetAsync(fs.pair_out[q], 0, sizeof(double) * 8 * np, s);
  emrt::note_launch(), k_pair_seq<<<dim3(152 * 8, fs.n), 256, 0, s>>>(rec, n, cap, n_tx, n_rx, fs);
  bool any_rx = false;
  for (uint32_t q = 0; q < fs.n; q++) any_rx = any_rx || fs.rx_out[q];
  if (any_rx)
    emrt::note_launch(), k_rx_power<<<dim3(ceil_div(n_rx, 256), fs.n), 256, 0, s>>>(n_tx, n_rx, tx_power_w, fs);
}

int adjoint_grid() { return 152 * 4; }

void launch_field_adjoint(const GeomView &g, MatView m, const uint32_t *rec, const uint32_t *n,
                          uint32_t cap, double freq, const double *dloss_dh, uint32_t n_rx,
                          double *contrib, double *grad_eps, double *grad_sigma, double *grad_tx,
                          Counters *ctr, cudaStream_t s) {
  emrt::note_launch(), k_field_tangents<<<adjoint_grid(), kAdjBlock, 0, s>>>(g, m, rec, n, cap, freq, dloss_dh, n_rx,
                                                        contrib, ctr);
  uint32_t n_par = 2 * m.n_mat + 3 * g.n_tx;
  emrt::note_launch(), k_grad_reduce<<<n_par, 256, 0, s>>>(g, m, rec, n, cap, contrib, grad_eps, grad_sigma, grad_tx);
}

}  // namespace emrt
