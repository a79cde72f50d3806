// Host launchers of the field, reduction and adjoint kernels.
#pragma once
#include "common.cuh"

namespace emrt {

struct MatView {
  const double *eps_r, *sigma, *gamma;
  uint32_t n_mat, const_gamma;
};

// device error bit raised by the field kernel when a path's amplitude,
// delay or Doppler is not finite (NaN or infinite material parameters or
// positions); a bit of Counters::err beside the ones of common.cuh
constexpr uint32_t ERR_NONFINITE = 32u;

// Frequencies of one channel evaluation and their outputs (rx_out[q] may be
// null).
constexpr uint32_t kMaxFreq = 8;
struct FreqSet {
  double f[kMaxFreq];
  double *path_out[kMaxFreq], *pair_out[kMaxFreq], *rx_out[kMaxFreq];
  uint32_t n;
};
// per frequency: per-path (Re a, Im a, tau, f_D) for min(*n, cap) canonical
// records, per (tx, rx) statistics (zeros for pairs without paths) and
// per-receiver powers; records must be in canonical order
void launch_channel(const GeomView &g, MatView m, const uint32_t *rec, const uint32_t *n,
                    uint32_t cap, const FreqSet &fs, uint32_t n_tx, uint32_t n_rx,
                    double tx_power_w, Counters *ctr, cudaStream_t s);
// adjoint: gradients w.r.t. eps_r [n_mat], sigma [n_mat], tx position
// [n_tx][3]; `partial` is per-path scratch of cap * (3 + 2 EMRT_MAX_DEPTH)
// doubles (tangent contributions), reduced per parameter in a fixed order; a
// non-finite amplitude or tangent raises ERR_NONFINITE in ctr->err
void launch_field_adjoint(const GeomView &g, MatView m, const uint32_t *rec, const uint32_t *n,
                          uint32_t cap, double freq, const double *dloss_dh, uint32_t n_rx,
                          double *partial, double *grad_eps, double *grad_sigma, double *grad_tx,
                          Counters *ctr, cudaStream_t s);
int adjoint_grid();
// Eq. 1 (normalised autocovariance of |h| over frames) and Eq. 2 (coherence
// time) of Sec. III-B
void launch_correlation(const double *h, uint32_t n_frames, uint32_t n_pairs, uint32_t max_lag,
                        double *R, cudaStream_t s);
void launch_coherence(const GeomView &g, double freq, double r_thr, double *tc, cudaStream_t s);
// Per-receiver re-discovery schedule: direct-path records of every pair,
// the due rule per receiver (flag[r] = 1 when due; state and los_ref updated)
// and the compaction of due ids (pos = exclusive scan of flag).
void launch_los_records(uint32_t n_tx, uint32_t n_rx, uint32_t *rec, cudaStream_t s);
void launch_schedule(const GeomView &g, const uint32_t *los, float4 *state, uint8_t *los_ref,
                     double freq, double r_thr, double dt, float d_seg, uint32_t max_interval,
                     uint32_t *flag, cudaStream_t s);
void launch_compact_ids(const uint32_t *flag, const uint32_t *pos, uint32_t n, uint32_t *ids,
                        cudaStream_t s);

}  // namespace emrt
