// Device-wide primitives with device-resident element counts: LSD radix sort
// of multi-word keys with a 32-bit payload, exclusive scan, stable
// compaction.  All launches use fixed grids (a multiple of the SM count), so
// they need no host synchronisation and can be captured in a CUDA graph.
#pragma once
#include "common.cuh"

namespace emrt {

constexpr int kPrimGrid = 2 * 152;   // blocks per primitive launch
constexpr int kPrimBlock = 256;

template <int W>
struct alignas(W == 1 ? 4 : (W == 2 ? 8 : 16)) KeyW {
  uint32_t w[W];
};

// Sorts (keys, vals)[0..*d_n) by the low `bits` bits of the W-word keys
// (word 0 least significant), stable.  Ping-pongs between (keys, vals) and
// (keys2, vals2); returns true when the result ends in (keys2, vals2).
// hist must hold 256 * kPrimGrid + 1 words.  max_n is a host-side upper
// bound of *d_n (the buffer capacity); it sets the grid size.
// first_pass > 0 skips the low 8 * first_pass bits: the result is then
// ordered by bits [8 * first_pass, bits) only.
template <int W>
bool radix_sort(const uint32_t *d_n, KeyW<W> *keys, uint32_t *vals,
                KeyW<W> *keys2, uint32_t *vals2, int bits, uint32_t *hist,
                cudaStream_t s, uint64_t max_n, int first_pass = 0);

// out[i] = sum_{k<i} in[i]; *d_total = sum (may alias nothing).  partial
// must hold kPrimGrid + 1 words.
void exclusive_scan(const uint32_t *d_n, const uint32_t *in, uint32_t *out,
                    uint32_t *d_total, uint32_t *partial, cudaStream_t s);

}  // namespace emrt
