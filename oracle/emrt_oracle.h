/*
 * CPU oracle for dynamic urban EM ray tracing (arXiv 2303.10521).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow FP64 restatement of the
 * method used to check the CUDA path; only the tests, the smoke check and
 * the benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or helper with the CUDA library.
 *
 * What it computes (paper passages in brackets):
 *  - shooting-and-bouncing discovery with reception spheres over a brute-force
 *    scan of every face polygon, no BVH [Sec. II-A: direct and reflected
 *    rays; BVH and path caching are accelerations, not part of the result];
 *  - image-method acceptance of face-ID sequences with occlusion tests
 *    [Sec. II-A, Sec. III-B: cached paths are kept while still valid];
 *  - per-path complex field: spreading, phase, polarimetric Fresnel
 *    reflection for complex permittivity, or the constant reflection
 *    coefficients of Table I, and the Doppler shift (Eq. 3 generalised to
 *    moving endpoints and moving reflectors) [Sec. III-C, Sec. IV];
 *  - exhaustive enumeration of every face sequence up to K reflections.
 *
 * All inputs are host arrays.  Face IDs: static faces 0..F_s-1, vehicle v
 * face j (j = -x,+x,-y,+y,-z,+z) is F_s + 6v + j.
 */
#ifndef EMRT_ORACLE_H
#define EMRT_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_DEPTH 4

typedef struct {
  int n_static_faces;
  const uint32_t *face_off;  /* [F_s+1] */
  const float *face_xyz;     /* [NV][3] */
  const uint32_t *face_mat;  /* [F_s] */
  int n_veh;
  const float *veh_half;     /* [V][3] */
  const float *veh_pos;      /* [V][3] box centres */
  const float *veh_vel;      /* [V][3] */
  uint32_t veh_mat;
  int n_rx;
  const float *rx_pos, *rx_vel; /* [R][3] */
  int n_tx;
  const float *tx_pos, *tx_vel; /* [X][3] */
  int n_mat;
  const double *eps_r, *sigma, *gamma; /* [M] */
  int const_gamma;           /* 1: Table I constant coefficients */
} orc_scene_desc;

/* candidate / path record as exchanged with Python */
typedef struct {
  uint32_t tx, rx, depth;
  uint32_t face[ORC_MAX_DEPTH];
  uint32_t ray;   /* ray index within its transmitter's ray set */
  uint32_t flag;  /* trace: 0 robust, 1 marginal, 2 marginal near-miss */
} orc_path;

typedef struct orc_scene_s *orc_scene;

orc_scene orc_scene_create(const orc_scene_desc *d);
void orc_scene_destroy(orc_scene s);
int orc_scene_n_faces(orc_scene s);
/* face plane as computed by the oracle (unit normal n, offset d: n.x = d) */
void orc_face_plane(orc_scene s, int f, double out[4]);

/* Fibonacci-sphere direction i of N, rounded once to float32. */
void orc_ray_dir(uint64_t n_rays, uint64_t i, float out[3]);

/* reception-sphere radius factor: r(L) = orc_radius_factor(N) * L */
double orc_radius_factor(uint64_t n_rays);

/* SBR discovery for every transmitter over rays offset + stride*j,
 * j < count.  Candidates (not deduplicated, in (tx, ray) order) go to
 * out[0..cap); the return value is the number produced (> cap means the
 * caller must retry with a larger buffer).  ray_marg[tx*count + j] receives
 * the first segment index whose outcome lies within the margin (255 when
 * none) and ray_segs the number of segments traced.
 * margin = eps_abs + eps_rel * (distance travelled). */
int64_t orc_trace(orc_scene s, uint64_t n_rays, int max_depth,
                  uint64_t offset, uint64_t stride, uint64_t count,
                  double eps_abs, double eps_rel, int n_threads,
                  orc_path *out, int64_t cap, uint8_t *ray_marg,
                  uint8_t *ray_segs);
/* Same, for an explicit list of ray indices (ray j of the traced set is
 * ray_idx[j]; candidates report j). */
int64_t orc_trace_list(orc_scene s, uint64_t n_rays, int max_depth,
                       const uint64_t *ray_idx, uint64_t count, double eps_abs,
                       double eps_rel, int n_threads, orc_path *out, int64_t cap,
                       uint8_t *ray_marg, uint8_t *ray_segs);

/* Image-method acceptance of n paths.  accepted[i] = 1 if valid; marginal[i]
 * bit0 = a reflection point or side test within the margin, bit1 = an
 * occlusion test within the margin.  points (optional) [n][ORC_MAX_DEPTH][3]
 * receives the reflection points. */
void orc_validate(orc_scene s, int64_t n, const orc_path *p, double eps_abs,
                  double eps_rel, int n_threads, uint8_t *accepted,
                  uint8_t *marginal, double *points);

/* Field of n accepted paths at frequency f (Hz):
 * a = (re, im) complex amplitude for 1 W transmit power, tau (s), fd (Hz). */
void orc_field(orc_scene s, int64_t n, const orc_path *p, double freq,
               int n_threads, double *a, double *tau, double *fd);

/* Fresnel coefficients (s and p, complex) for permittivity eps (complex)
 * and incidence cosine cos_t. */
void orc_fresnel(double eps_re, double eps_im, double cos_t, double out[4]);

/* Every valid path with up to max_depth reflections (all face sequences
 * without immediate repeats).  Returns the count (> cap: retry). */
int64_t orc_enumerate(orc_scene s, int max_depth, int n_threads,
                      orc_path *out, int64_t cap);

#ifdef __cplusplus
}
#endif
#endif
