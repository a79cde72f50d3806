// Host launchers of the field, reduction and adjoint kernels.
#pragma once
#include "common.cuh"

namespace emrt {

struct MatView {
  const double *eps_r, *sigma, *gamma;
  uint32_t n_mat, const_gamma;
};

// per-path (Re a, Im a, tau, f_D) for min(*n, cap) canonical records
void launch_field(const GeomView &g, MatView m, const uint32_t *rec, const uint32_t *n,
                  uint32_t cap, double freq, double *path_out, cudaStream_t s);
// per (tx, rx) statistics and per-receiver powers; seg_begin/seg_end are
// scratch of n_tx * n_rx words each
void launch_reduce(const uint32_t *rec, const uint32_t *n, uint32_t cap, const double *path_out,
                   uint32_t n_tx, uint32_t n_rx, double tx_power_w, uint32_t *seg_begin,
                   uint32_t *seg_end, double *pair_out, double *rx_out, cudaStream_t s);
// adjoint: grad (2 n_mat + 3 n_tx doubles, layout eps | sigma | tx xyz),
// partial: per-block scratch of grid * (2 n_mat + 3 n_tx) doubles
void launch_field_adjoint(const GeomView &g, MatView m, const uint32_t *rec, const uint32_t *n,
                          uint32_t cap, double freq, const double *dloss_dh, uint32_t n_rx,
                          double *partial, double *grad_eps, double *grad_sigma, double *grad_tx,
                          cudaStream_t s);
int adjoint_grid();

}  // namespace emrt
