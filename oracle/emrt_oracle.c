/*
 * CPU oracle for dynamic urban EM ray tracing (arXiv 2303.10521).
 *
 * TEST INFRASTRUCTURE ONLY: plain FP64 restatement of the method used to
 * check the CUDA path.  Brute force over every face polygon; no BVH, no
 * sorting, no caching.  Only tests, the smoke check and the benchmark's CPU
 * baseline may call it.  Shares no code with the CUDA library.
 *
 * Readings of points the paper leaves open (each applied identically here
 * and stated in the design notes):
 *  - a face is a convex planar polygon; hits and reflection points are
 *    tested against the polygon, boundary inclusive;
 *  - rays leaving a face ignore that face for their next segment;
 *  - a closest-hit tie goes to the lower face ID;
 *  - the reception radius is r(L) = 1.25 * sqrt(8 pi / (3 sqrt(3) N)) * L,
 *    the hexagonal covering angle of N directions widened by the measured
 *    excess of the Fibonacci lattice near its poles; a receiver is detected
 *    when the traced segment passes within r(L) of it (L at the segment
 *    point nearest to the receiver);
 *  - antennas are ideal omnidirectional and vertically polarised:
 *    p(k) = normalise(z - (z.k) k);
 *  - time convention exp(+j w t): propagation is exp(-j k L);
 *  - Table I constant mode: Gamma_s = -gamma, Gamma_p = +gamma (a scaled
 *    perfect conductor).
 */
#include "emrt_oracle.h"

#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define C0 299792458.0
#define EPS0 8.8541878128e-12

typedef struct { double x, y, z; } v3;
static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double norm(v3 a) { return sqrt(dot(a, a)); }
static v3 unit(v3 a) { return scl(a, 1.0 / norm(a)); }
static v3 ld3(const float *p) { return mk(p[0], p[1], p[2]); }

typedef struct {
  int nv;
  v3 *v;        /* polygon vertices, CCW about n */
  v3 n;         /* unit normal */
  double d;     /* plane offset: n.x = d */
  int mat;
  v3 vel;       /* velocity of the face (vehicles), zero for static */
} face_t;

struct orc_scene_s {
  int nf, nfs;
  face_t *f;
  v3 *vstore;
  int nrx, ntx;
  v3 *rx, *rxv, *tx, *txv;
  int nmat;
  double *eps, *sig, *gam;
  int const_gamma;
};

/* Newell's method: normal of a planar polygon, then offset from the mean
 * vertex. */
static void face_plane(face_t *F) {
  v3 n = mk(0, 0, 0), c = mk(0, 0, 0);
  for (int i = 0; i < F->nv; i++) {
    v3 a = F->v[i], b = F->v[(i + 1) % F->nv];
    n.x += (a.y - b.y) * (a.z + b.z);
    n.y += (a.z - b.z) * (a.x + b.x);
    n.z += (a.x - b.x) * (a.y + b.y);
    c = add(c, a);
  }
  F->n = unit(n);
  F->d = dot(F->n, scl(c, 1.0 / F->nv));
}

orc_scene orc_scene_create(const orc_scene_desc *D) {
  orc_scene s = (orc_scene)calloc(1, sizeof(*s));
  s->nfs = D->n_static_faces;
  s->nf = D->n_static_faces + 6 * D->n_veh;
  s->f = (face_t *)calloc(s->nf ? s->nf : 1, sizeof(face_t));
  int nvs = D->n_static_faces ? (int)D->face_off[D->n_static_faces] : 0;
  s->vstore = (v3 *)calloc(nvs + 24 * D->n_veh + 1, sizeof(v3));
  v3 *vp = s->vstore;
  for (int f = 0; f < D->n_static_faces; f++) {
    face_t *F = &s->f[f];
    F->nv = (int)(D->face_off[f + 1] - D->face_off[f]);
    F->v = vp;
    for (int i = 0; i < F->nv; i++) vp[i] = ld3(D->face_xyz + 3 * (D->face_off[f] + i));
    vp += F->nv;
    F->mat = (int)D->face_mat[f];
    F->vel = mk(0, 0, 0);
    face_plane(F);
  }
  for (int v = 0; v < D->n_veh; v++) {
    /* box corners in float32 arithmetic, as the scene defines them */
    float lo[3], hi[3];
    for (int k = 0; k < 3; k++) {
      lo[k] = D->veh_pos[3 * v + k] - D->veh_half[3 * v + k];
      hi[k] = D->veh_pos[3 * v + k] + D->veh_half[3 * v + k];
    }
    double x0 = lo[0], y0 = lo[1], z0 = lo[2], x1 = hi[0], y1 = hi[1], z1 = hi[2];
    v3 q[6][4] = {
        {{x0, y0, z0}, {x0, y0, z1}, {x0, y1, z1}, {x0, y1, z0}}, /* -x */
        {{x1, y0, z0}, {x1, y1, z0}, {x1, y1, z1}, {x1, y0, z1}}, /* +x */
        {{x0, y0, z0}, {x1, y0, z0}, {x1, y0, z1}, {x0, y0, z1}}, /* -y */
        {{x0, y1, z0}, {x0, y1, z1}, {x1, y1, z1}, {x1, y1, z0}}, /* +y */
        {{x0, y0, z0}, {x0, y1, z0}, {x1, y1, z0}, {x1, y0, z0}}, /* -z */
        {{x0, y0, z1}, {x1, y0, z1}, {x1, y1, z1}, {x0, y1, z1}}, /* +z */
    };
    for (int j = 0; j < 6; j++) {
      face_t *F = &s->f[s->nfs + 6 * v + j];
      F->nv = 4;
      F->v = vp;
      for (int i = 0; i < 4; i++) vp[i] = q[j][i];
      vp += 4;
      F->mat = (int)D->veh_mat;
      F->vel = ld3(D->veh_vel + 3 * v);
      face_plane(F);
    }
  }
  s->nrx = D->n_rx;
  s->ntx = D->n_tx;
  s->rx = (v3 *)calloc(D->n_rx + 1, sizeof(v3));
  s->rxv = (v3 *)calloc(D->n_rx + 1, sizeof(v3));
  s->tx = (v3 *)calloc(D->n_tx + 1, sizeof(v3));
  s->txv = (v3 *)calloc(D->n_tx + 1, sizeof(v3));
  for (int i = 0; i < D->n_rx; i++) {
    s->rx[i] = ld3(D->rx_pos + 3 * i);
    s->rxv[i] = ld3(D->rx_vel + 3 * i);
  }
  for (int i = 0; i < D->n_tx; i++) {
    s->tx[i] = ld3(D->tx_pos + 3 * i);
    s->txv[i] = ld3(D->tx_vel + 3 * i);
  }
  s->nmat = D->n_mat;
  s->eps = (double *)malloc(sizeof(double) * (D->n_mat + 1));
  s->sig = (double *)malloc(sizeof(double) * (D->n_mat + 1));
  s->gam = (double *)malloc(sizeof(double) * (D->n_mat + 1));
  memcpy(s->eps, D->eps_r, sizeof(double) * D->n_mat);
  memcpy(s->sig, D->sigma, sizeof(double) * D->n_mat);
  memcpy(s->gam, D->gamma, sizeof(double) * D->n_mat);
  s->const_gamma = D->const_gamma;
  return s;
}

void orc_scene_destroy(orc_scene s) {
  if (!s) return;
  free(s->f); free(s->vstore); free(s->rx); free(s->rxv); free(s->tx);
  free(s->txv); free(s->eps); free(s->sig); free(s->gam); free(s);
}

int orc_scene_n_faces(orc_scene s) { return s->nf; }

void orc_face_plane(orc_scene s, int f, double out[4]) {
  out[0] = s->f[f].n.x; out[1] = s->f[f].n.y; out[2] = s->f[f].n.z;
  out[3] = s->f[f].d;
}

/* Signed distance of a point on the face plane to the polygon boundary:
 * >= 0 inside (boundary inclusive), < 0 outside.  Outside, its magnitude is
 * at most the true distance, which keeps the margin test conservative. */
static double inside_margin(const face_t *F, v3 p) {
  double m = INFINITY;
  for (int i = 0; i < F->nv; i++) {
    v3 a = F->v[i], b = F->v[(i + 1) % F->nv];
    v3 e = sub(b, a);
    double sd = dot(cross(e, sub(p, a)), F->n) / norm(e);
    if (sd < m) m = sd;
  }
  return m;
}

/* ------------------------------------------------------------------ */
/* thread pool over index chunks                                       */
/* ------------------------------------------------------------------ */
typedef void (*chunk_fn)(void *ctx, int64_t chunk);
typedef struct { chunk_fn fn; void *ctx; int64_t n; int64_t next; pthread_mutex_t mu; } pool_t;

static void *pool_worker(void *arg) {
  pool_t *P = (pool_t *)arg;
  for (;;) {
    pthread_mutex_lock(&P->mu);
    int64_t c = P->next++;
    pthread_mutex_unlock(&P->mu);
    if (c >= P->n) break;
    P->fn(P->ctx, c);
  }
  return NULL;
}

static void run_chunks(int64_t n_chunks, int n_threads, chunk_fn fn, void *ctx) {
  pool_t P;
  P.fn = fn; P.ctx = ctx; P.n = n_chunks; P.next = 0;
  pthread_mutex_init(&P.mu, NULL);
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  for (int i = 0; i < n_threads; i++) pthread_create(&th[i], NULL, pool_worker, &P);
  for (int i = 0; i < n_threads; i++) pthread_join(th[i], NULL);
  pthread_mutex_destroy(&P.mu);
}

/* ------------------------------------------------------------------ */
/* ray directions and reception radius                                 */
/* ------------------------------------------------------------------ */
void orc_ray_dir(uint64_t n, uint64_t i, float out[3]) {
  /* Fibonacci sphere: uniform steps in z, golden-angle steps in azimuth */
  double z = 1.0 - (2.0 * (double)i + 1.0) / (double)n;
  double rho = sqrt(fmax(0.0, 1.0 - z * z));
  double g = (3.0 - sqrt(5.0)) / 2.0;
  double t = (double)i * g;
  double phi = 2.0 * M_PI * (t - floor(t));
  out[0] = (float)(rho * cos(phi));
  out[1] = (float)(rho * sin(phi));
  out[2] = (float)z;
}

double orc_radius_factor(uint64_t n) {
  return 1.25 * sqrt(8.0 * M_PI / (3.0 * sqrt(3.0) * (double)n));
}

/* ------------------------------------------------------------------ */
/* SBR discovery                                                        */
/* ------------------------------------------------------------------ */
typedef struct { orc_path *p; int64_t n, cap; } pbuf;
static void pb_push(pbuf *b, const orc_path *r) {
  if (b->n == b->cap) {
    b->cap = b->cap ? 2 * b->cap : 16;
    b->p = (orc_path *)realloc(b->p, sizeof(orc_path) * b->cap);
  }
  b->p[b->n++] = *r;
}

#define TRACE_CHUNK 64
typedef struct {
  orc_scene s;
  uint64_t n_rays, offset, stride, count;
  const uint64_t *idx;  /* explicit ray list, or NULL */
  int K;
  double eps_abs, eps_rel, kappa;
  pbuf *bufs;  /* per chunk */
  uint8_t *marg, *segs;
} trace_ctx;

static void trace_one(trace_ctx *C, int tx, uint64_t j, pbuf *out, uint8_t *marg_out,
                      uint8_t *segs_out) {
  orc_scene s = C->s;
  uint64_t idx = C->idx ? C->idx[j] : C->offset + C->stride * j;
  float df[3];
  orc_ray_dir(C->n_rays, idx, df);
  v3 d = unit(ld3(df));
  v3 o = s->tx[tx];
  double Lacc = 0.0;
  int prev = -1;
  uint32_t faces[ORC_MAX_DEPTH];
  int first_marg = 255, nseg = 0;
  for (int b = 0; b <= C->K; b++) {
    nseg++;
    double eps = C->eps_abs + C->eps_rel * Lacc;
    double best_t = INFINITY;
    int best_f = -1;
    double near_t = INFINITY;  /* nearest face event within the margin */
    for (int f = 0; f < s->nf; f++) {
      if (f == prev) continue;
      const face_t *F = &s->f[f];
      double den = dot(F->n, d);
      if (den == 0.0) continue;
      double t = (F->d - dot(F->n, o)) / den;
      if (!(t > 0.0)) continue;
      double m = inside_margin(F, add(o, scl(d, t)));
      if (m >= 0.0 && (t < best_t || (t == best_t && f < best_f))) {
        best_t = t;
        best_f = f;
      }
      double e = eps + C->eps_rel * t;
      if (fabs(m) < e && t < near_t) near_t = t;
    }
    /* a second face hit at (almost) the same distance is a coincidence */
    if (best_f >= 0) {
      for (int f = 0; f < s->nf; f++) {
        if (f == prev || f == best_f) continue;
        const face_t *F = &s->f[f];
        double den = dot(F->n, d);
        if (den == 0.0) continue;
        double t = (F->d - dot(F->n, o)) / den;
        if (fabs(t - best_t) < eps + C->eps_rel * best_t &&
            inside_margin(F, add(o, scl(d, t))) >= -(eps + C->eps_rel * best_t))
          near_t = fmin(near_t, t);
      }
    }
    double e_end = eps + C->eps_rel * (isfinite(best_t) ? best_t : 0.0);
    int seg_marg = isfinite(near_t) && near_t <= best_t + e_end;
    if (seg_marg && first_marg == 255) first_marg = b;
    /* reception spheres: a receiver is detected when the traced segment
     * [0, best_t] (a ray when nothing is hit) passes within r(L) of it, with
     * L the unfolded length at the segment point nearest to the receiver */
    for (int r = 0; r < s->nrx; r++) {
      v3 w = sub(s->rx[r], o);
      double sp = dot(w, d);
      double sc = fmin(fmax(sp, 0.0), best_t);
      double dist = norm(sub(w, scl(d, sc)));
      double rad = C->kappa * (Lacc + sc);
      double e = eps + C->eps_rel * sc;
      int inside = dist <= rad;
      int near_sphere = fabs(dist - rad) < e;
      if (!inside && !near_sphere) continue;
      orc_path rec;
      memset(&rec, 0, sizeof(rec));
      rec.tx = (uint32_t)tx;
      rec.rx = (uint32_t)r;
      rec.depth = (uint32_t)b;
      for (int k = 0; k < b; k++) rec.face[k] = faces[k];
      for (int k = b; k < ORC_MAX_DEPTH; k++) rec.face[k] = 0xffffffffu;
      rec.ray = (uint32_t)j;
      if (!inside) rec.flag = 2;
      else if (near_sphere || first_marg != 255) rec.flag = 1;
      else rec.flag = 0;
      pb_push(out, &rec);
    }
    if (best_f < 0 || b == C->K) break;
    /* specular reflection at the hit point */
    const face_t *F = &s->f[best_f];
    o = add(o, scl(d, best_t));
    d = unit(sub(d, scl(F->n, 2.0 * dot(d, F->n))));
    Lacc += best_t;
    faces[b] = (uint32_t)best_f;
    prev = best_f;
  }
  *marg_out = (uint8_t)first_marg;
  *segs_out = (uint8_t)nseg;
}

static void trace_chunk(void *ctx, int64_t c) {
  trace_ctx *C = (trace_ctx *)ctx;
  uint64_t per_tx = (C->count + TRACE_CHUNK - 1) / TRACE_CHUNK;
  int tx = (int)(c / per_tx);
  uint64_t j0 = (uint64_t)(c % per_tx) * TRACE_CHUNK;
  uint64_t j1 = j0 + TRACE_CHUNK;
  if (j1 > C->count) j1 = C->count;
  for (uint64_t j = j0; j < j1; j++)
    trace_one(C, tx, j, &C->bufs[c], &C->marg[tx * C->count + j],
              &C->segs[tx * C->count + j]);
}

static int64_t trace_impl(orc_scene s, uint64_t n_rays, int max_depth, uint64_t offset,
                          uint64_t stride, const uint64_t *idx, uint64_t count, double eps_abs,
                          double eps_rel, int n_threads, orc_path *out, int64_t cap,
                          uint8_t *ray_marg, uint8_t *ray_segs) {
  trace_ctx C;
  C.s = s; C.n_rays = n_rays; C.offset = offset; C.stride = stride; C.idx = idx;
  C.count = count; C.K = max_depth; C.eps_abs = eps_abs; C.eps_rel = eps_rel;
  C.kappa = orc_radius_factor(n_rays);
  C.marg = ray_marg; C.segs = ray_segs;
  uint64_t per_tx = (count + TRACE_CHUNK - 1) / TRACE_CHUNK;
  int64_t nch = (int64_t)(per_tx * s->ntx);
  C.bufs = (pbuf *)calloc(nch + 1, sizeof(pbuf));
  run_chunks(nch, n_threads, trace_chunk, &C);
  int64_t total = 0;
  for (int64_t c = 0; c < nch; c++) {
    for (int64_t i = 0; i < C.bufs[c].n; i++) {
      if (total < cap) out[total] = C.bufs[c].p[i];
      total++;
    }
    free(C.bufs[c].p);
  }
  free(C.bufs);
  return total;
}

int64_t orc_trace(orc_scene s, uint64_t n_rays, int max_depth, uint64_t offset,
                  uint64_t stride, uint64_t count, double eps_abs, double eps_rel,
                  int n_threads, orc_path *out, int64_t cap, uint8_t *ray_marg,
                  uint8_t *ray_segs) {
  return trace_impl(s, n_rays, max_depth, offset, stride, NULL, count, eps_abs, eps_rel,
                    n_threads, out, cap, ray_marg, ray_segs);
}

int64_t orc_trace_list(orc_scene s, uint64_t n_rays, int max_depth, const uint64_t *ray_idx,
                       uint64_t count, double eps_abs, double eps_rel, int n_threads,
                       orc_path *out, int64_t cap, uint8_t *ray_marg, uint8_t *ray_segs) {
  return trace_impl(s, n_rays, max_depth, 0, 1, ray_idx, count, eps_abs, eps_rel, n_threads,
                    out, cap, ray_marg, ray_segs);
}

/* ------------------------------------------------------------------ */
/* image method                                                         */
/* ------------------------------------------------------------------ */
static v3 mirror(v3 p, const face_t *F) {
  return sub(p, scl(F->n, 2.0 * (dot(F->n, p) - F->d)));
}

/* Reflection points of a face sequence by the image method.  Q[0] = Tx,
 * Q[1..k] reflection points, Q[k+1] = Rx.  Returns 0 when a segment does
 * not cross its face plane inside (0, 1); *inface_m gets the smallest
 * polygon margin of the points and *side_m the smallest distance of the
 * neighbouring points to the face planes (negative: wrong side). */
static int image_points(orc_scene s, const orc_path *p, v3 *Q, double *inface_m,
                        double *side_m, double *t_m) {
  int k = (int)p->depth;
  v3 Im[ORC_MAX_DEPTH + 1];
  Im[0] = s->tx[p->tx];
  for (int j = 1; j <= k; j++) Im[j] = mirror(Im[j - 1], &s->f[p->face[j - 1]]);
  Q[0] = s->tx[p->tx];
  Q[k + 1] = s->rx[p->rx];
  *inface_m = INFINITY;
  *side_m = INFINITY;
  *t_m = INFINITY;
  for (int j = k; j >= 1; j--) {
    const face_t *F = &s->f[p->face[j - 1]];
    v3 D = sub(Q[j + 1], Im[j]);
    double den = dot(F->n, D);
    if (den == 0.0) return 0;
    double t = (F->d - dot(F->n, Im[j])) / den;
    if (!(t > 0.0 && t < 1.0)) return 0;
    *t_m = fmin(*t_m, fmin(t, 1.0 - t) * norm(D));
    Q[j] = add(Im[j], scl(D, t));
    *inface_m = fmin(*inface_m, inside_margin(F, Q[j]));
  }
  for (int j = 1; j <= k; j++) {
    const face_t *F = &s->f[p->face[j - 1]];
    double a = dot(F->n, Q[j - 1]) - F->d;
    double b = dot(F->n, Q[j + 1]) - F->d;
    /* same strict side: a genuine specular bounce */
    double m = (a > 0) == (b > 0) ? fmin(fabs(a), fabs(b)) : -fmin(fabs(a), fabs(b));
    if (a == 0.0 || b == 0.0) m = 0.0;
    *side_m = fmin(*side_m, m);
  }
  return 1;
}

/* Occlusion of the segment A->B by any face other than ex0, ex1.
 * Returns 1 when blocked; *marg is set when a face crossing lies within the
 * margin of its polygon boundary or of the segment ends. */
static int occluded(orc_scene s, v3 A, v3 B, int ex0, int ex1, double eps, int *marg) {
  v3 D = sub(B, A);
  double len = norm(D);
  int hit = 0;
  for (int g = 0; g < s->nf; g++) {
    if (g == ex0 || g == ex1) continue;
    const face_t *F = &s->f[g];
    double den = dot(F->n, D);
    if (den == 0.0) continue;
    double t = (F->d - dot(F->n, A)) / den;
    double te = eps / len;
    if (t <= -te || t >= 1.0 + te) continue;
    double m = inside_margin(F, add(A, scl(D, t)));
    int strict = t > 0.0 && t < 1.0;
    if (strict && m >= 0.0) hit = 1;
    if (fabs(m) < eps) *marg = 1;
    if (m >= 0.0 && (t * len < eps || (1.0 - t) * len < eps)) *marg = 1;
  }
  return hit;
}

static int validate_one(orc_scene s, const orc_path *p, double eps_abs, double eps_rel,
                        uint8_t *marg, v3 *Q) {
  int k = (int)p->depth;
  *marg = 0;
  if (k > ORC_MAX_DEPTH) return 0;
  for (int j = 0; j < k; j++) {
    if ((int)p->face[j] >= s->nf) return 0;
    if (j > 0 && p->face[j] == p->face[j - 1]) return 0;
  }
  double fm, sm, tm;
  if (!image_points(s, p, Q, &fm, &sm, &tm)) return 0;
  double Ltot = 0.0;
  for (int j = 0; j <= k; j++) Ltot += norm(sub(Q[j + 1], Q[j]));
  double eps = eps_abs + eps_rel * Ltot;
  if (fabs(fm) < eps || fabs(sm) < eps || tm < eps) *marg |= 1;
  int ok = fm >= 0.0 && sm > 0.0;
  int om = 0;
  for (int j = 0; j <= k; j++) {
    int e0 = j >= 1 ? (int)p->face[j - 1] : -1;
    int e1 = j < k ? (int)p->face[j] : -1;
    if (occluded(s, Q[j], Q[j + 1], e0, e1, eps, &om)) ok = 0;
  }
  if (om) *marg |= 2;
  return ok;
}

typedef struct {
  orc_scene s;
  const orc_path *p;
  int64_t n;
  double ea, er;
  uint8_t *acc, *marg;
  double *pts;
} val_ctx;

#define VAL_CHUNK 256
static void val_chunk(void *ctx, int64_t c) {
  val_ctx *C = (val_ctx *)ctx;
  int64_t i1 = (c + 1) * VAL_CHUNK;
  if (i1 > C->n) i1 = C->n;
  for (int64_t i = c * VAL_CHUNK; i < i1; i++) {
    v3 Q[ORC_MAX_DEPTH + 2];
    uint8_t m;
    C->acc[i] = (uint8_t)validate_one(C->s, &C->p[i], C->ea, C->er, &m, Q);
    C->marg[i] = m;
    if (C->pts) {
      for (int j = 0; j < ORC_MAX_DEPTH; j++) {
        double *o = C->pts + (i * ORC_MAX_DEPTH + j) * 3;
        if (j < (int)C->p[i].depth && C->acc[i]) {
          o[0] = Q[j + 1].x; o[1] = Q[j + 1].y; o[2] = Q[j + 1].z;
        } else {
          o[0] = o[1] = o[2] = NAN;
        }
      }
    }
  }
}

void orc_validate(orc_scene s, int64_t n, const orc_path *p, double eps_abs,
                  double eps_rel, int n_threads, uint8_t *accepted, uint8_t *marginal,
                  double *points) {
  val_ctx C = {s, p, n, eps_abs, eps_rel, accepted, marginal, points};
  run_chunks((n + VAL_CHUNK - 1) / VAL_CHUNK, n_threads, val_chunk, &C);
}

/* ------------------------------------------------------------------ */
/* field                                                                */
/* ------------------------------------------------------------------ */
void orc_fresnel(double eps_re, double eps_im, double cos_t, double out[4]) {
  double complex ec = eps_re + I * eps_im;
  double sin2 = 1.0 - cos_t * cos_t;
  double complex root = csqrt(ec - sin2);
  double complex gs = (cos_t - root) / (cos_t + root);
  double complex gp = (ec * cos_t - root) / (ec * cos_t + root);
  out[0] = creal(gs); out[1] = cimag(gs); out[2] = creal(gp); out[3] = cimag(gp);
}

/* vertical transverse polarisation of an ideal omnidirectional antenna */
static v3 polar(v3 k) {
  v3 z = mk(0, 0, 1);
  v3 p = sub(z, scl(k, dot(z, k)));
  double n = norm(p);
  if (n < 1e-12) return mk(1, 0, 0);
  return scl(p, 1.0 / n);
}

typedef struct { double complex x, y, z; } c3;
static double complex cdotr(c3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

static void field_one(orc_scene s, const orc_path *p, double f, double *a, double *tau,
                      double *fd) {
  int k = (int)p->depth;
  v3 Q[ORC_MAX_DEPTH + 2];
  double fm, sm, tm;
  image_points(s, p, Q, &fm, &sm, &tm);
  v3 kh[ORC_MAX_DEPTH + 1];
  double L = 0.0;
  for (int j = 0; j <= k; j++) {
    v3 D = sub(Q[j + 1], Q[j]);
    double l = norm(D);
    L += l;
    kh[j] = scl(D, 1.0 / l);
  }
  double lam = C0 / f;
  v3 p0 = polar(kh[0]);
  c3 E = {p0.x, p0.y, p0.z};
  for (int j = 1; j <= k; j++) {
    const face_t *F = &s->f[p->face[j - 1]];
    v3 kin = kh[j - 1], kout = kh[j];
    double cos_t = fabs(dot(kin, F->n));
    v3 sv = cross(kin, F->n);
    if (norm(sv) < 1e-12) {  /* normal incidence: any s orthogonal to kin */
      sv = cross(kin, mk(1, 0, 0));
      if (norm(sv) < 1e-6) sv = cross(kin, mk(0, 1, 0));
    }
    sv = unit(sv);
    v3 pin = cross(sv, kin), pout = cross(sv, kout);
    double complex gs, gp;
    if (s->const_gamma) {
      gs = -s->gam[F->mat];
      gp = s->gam[F->mat];
    } else {
      double g[4];
      double eim = -s->sig[F->mat] / (2.0 * M_PI * f * EPS0);
      orc_fresnel(s->eps[F->mat], eim, cos_t, g);
      gs = g[0] + I * g[1];
      gp = g[2] + I * g[3];
    }
    double complex es = cdotr(E, sv), ep = cdotr(E, pin);
    c3 En;
    En.x = gs * es * sv.x + gp * ep * pout.x;
    En.y = gs * es * sv.y + gp * ep * pout.y;
    En.z = gs * es * sv.z + gp * ep * pout.z;
    E = En;
  }
  double complex rcv = cdotr(E, polar(kh[k]));
  double cyc = L / lam;
  double ph = -2.0 * M_PI * (cyc - floor(cyc));
  double complex amp = (lam / (4.0 * M_PI * L)) * cexp(I * ph) * rcv;
  a[0] = creal(amp);
  a[1] = cimag(amp);
  *tau = L / C0;
  /* rate of change of the unfolded length */
  double dL = -dot(s->txv[p->tx], kh[0]) + dot(s->rxv[p->rx], kh[k]);
  for (int j = 1; j <= k; j++)
    dL += dot(s->f[p->face[j - 1]].vel, sub(kh[j - 1], kh[j]));
  *fd = -(f / C0) * dL;
}

typedef struct {
  orc_scene s; const orc_path *p; int64_t n; double f;
  double *a, *tau, *fd;
} field_ctx;

static void field_chunk(void *ctx, int64_t c) {
  field_ctx *C = (field_ctx *)ctx;
  int64_t i1 = (c + 1) * VAL_CHUNK;
  if (i1 > C->n) i1 = C->n;
  for (int64_t i = c * VAL_CHUNK; i < i1; i++)
    field_one(C->s, &C->p[i], C->f, C->a + 2 * i, C->tau + i, C->fd + i);
}

void orc_field(orc_scene s, int64_t n, const orc_path *p, double freq, int n_threads,
               double *a, double *tau, double *fd) {
  field_ctx C = {s, p, n, freq, a, tau, fd};
  run_chunks((n + VAL_CHUNK - 1) / VAL_CHUNK, n_threads, field_chunk, &C);
}

/* ------------------------------------------------------------------ */
/* exhaustive enumeration                                              */
/* ------------------------------------------------------------------ */
typedef struct { orc_scene s; int K; pbuf *bufs; } enum_ctx;

static void enum_pair(void *ctx, int64_t c) {
  enum_ctx *C = (enum_ctx *)ctx;
  orc_scene s = C->s;
  orc_path p;
  memset(&p, 0, sizeof(p));
  p.tx = (uint32_t)(c / s->nrx);
  p.rx = (uint32_t)(c % s->nrx);
  for (int k = 0; k <= C->K; k++) {
    if (k > 0 && s->nf == 0) break;
    /* odometer over face sequences of length k */
    int idx[ORC_MAX_DEPTH] = {0, 0, 0, 0};
    for (;;) {
      int ok = 1;
      for (int j = 1; j < k; j++) if (idx[j] == idx[j - 1]) ok = 0;
      if (ok) {
        p.depth = (uint32_t)k;
        for (int j = 0; j < ORC_MAX_DEPTH; j++)
          p.face[j] = j < k ? (uint32_t)idx[j] : 0xffffffffu;
        v3 Q[ORC_MAX_DEPTH + 2];
        uint8_t m;
        if (validate_one(s, &p, 0.0, 0.0, &m, Q)) pb_push(&C->bufs[c], &p);
      }
      int j = k - 1;
      while (j >= 0 && ++idx[j] == s->nf) idx[j--] = 0;
      if (j < 0) break;
    }
  }
}

int64_t orc_enumerate(orc_scene s, int max_depth, int n_threads, orc_path *out,
                      int64_t cap) {
  int64_t npairs = (int64_t)s->ntx * s->nrx;
  enum_ctx C = {s, max_depth, (pbuf *)calloc(npairs + 1, sizeof(pbuf))};
  run_chunks(npairs, n_threads, enum_pair, &C);
  int64_t total = 0;
  for (int64_t c = 0; c < npairs; c++) {
    for (int64_t i = 0; i < C.bufs[c].n; i++) {
      if (total < cap) out[total] = C.bufs[c].p[i];
      total++;
    }
    free(C.bufs[c].p);
  }
  free(C.bufs);
  return total;
}
