// LSD radix sort, exclusive scan (fixed grids, device-side counts).
#include <algorithm>

#include "prims.cuh"

namespace emrt {

namespace {

__device__ inline void block_range(uint32_t n, uint32_t &lo, uint32_t &hi) {
  // contiguous chunk per block, a multiple of the block size
  uint32_t per = (n + gridDim.x - 1) / gridDim.x;
  per = (per + kPrimBlock - 1) / kPrimBlock * kPrimBlock;
  lo = min(n, blockIdx.x * per);
  hi = min(n, lo + per);
}

template <int W>
__device__ inline uint32_t digit_of(const KeyW<W> &k, int pass) {
  return (k.w[pass >> 2] >> ((pass & 3) * 8)) & 255u;
}

template <int W>
__global__ void __launch_bounds__(kPrimBlock) k_hist(const uint32_t *d_n, const KeyW<W> *keys,
                                                     int pass, uint32_t *hist) {
  __shared__ uint32_t sh[256];
  sh[threadIdx.x] = 0;
  __syncthreads();
  uint32_t lo, hi;
  block_range(*d_n, lo, hi);
  for (uint32_t i = lo + threadIdx.x; i < hi; i += kPrimBlock)
    atomicAdd(&sh[digit_of<W>(keys[i], pass)], 1u);
  __syncthreads();
  hist[blockIdx.x * 256 + threadIdx.x] = sh[threadIdx.x];
}

// Digit offsets from the block-major histogram hist[b][d] (G blocks):
// offs[b][d] = sum_{d' < d} total[d'] + sum_{b' < b} hist[b'][d].  1024
// threads: four groups of 256 (one thread per digit) split the rows, so
// every row access is a coalesced 1 KB load.  Only the rows of blocks that
// received keys (block_range's split of *d_n over G blocks) are read and
// written; the others scatter nothing.
__global__ void __launch_bounds__(1024) k_digit_offsets(const uint32_t *d_n, uint32_t *hist,
                                                        int G) {
  __shared__ uint32_t part[4][256];
  __shared__ uint32_t base[256];
  {
    const uint32_t n = *d_n;
    uint32_t per = (n + G - 1) / G;
    per = (per + kPrimBlock - 1) / kPrimBlock * kPrimBlock;
    G = per ? min(G, (int)((n + per - 1) / per)) : 0;
  }
  const int d = threadIdx.x & 255, grp = threadIdx.x >> 8;
  const int per = (G + 3) / 4, b0 = min(G, grp * per), b1 = min(G, b0 + per);
  uint32_t s = 0;
#pragma unroll 4
  for (int b = b0; b < b1; b++) s += hist[b * 256 + d];
  part[grp][d] = s;
  __syncthreads();
  if (grp == 0) base[d] = part[0][d] + part[1][d] + part[2][d] + part[3][d];
  __syncthreads();
  for (int off = 1; off < 256; off <<= 1) {
    uint32_t t = (grp == 0 && d >= off) ? base[d - off] : 0;
    __syncthreads();
    if (grp == 0) base[d] += t;
    __syncthreads();
  }
  uint32_t run = base[d] - (part[0][d] + part[1][d] + part[2][d] + part[3][d]);
  for (int q = 0; q < grp; q++) run += part[q][d];
#pragma unroll 4
  for (int b = b0; b < b1; b++) {
    uint32_t t = hist[b * 256 + d];
    hist[b * 256 + d] = run;
    run += t;
  }
}

// exclusive scan of n (<= a few 100k) words in one block of 1024 threads
__global__ void __launch_bounds__(1024) k_scan_single(uint32_t *v, uint32_t n, uint32_t *total) {
  __shared__ uint32_t part[1024];
  uint32_t per = (n + 1023) / 1024;
  uint32_t lo = min(n, threadIdx.x * per), hi = min(n, lo + per);
  uint32_t s = 0;
  for (uint32_t i = lo; i < hi; i++) s += v[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    uint32_t t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += t;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - s;
  for (uint32_t i = lo; i < hi; i++) {
    uint32_t t = v[i];
    v[i] = run;
    run += t;
  }
  if (threadIdx.x == 1023 && total) *total = part[1023];
}

// Stable scatter of one radix pass.  The block's key range (block_range) is
// processed in tiles of kPrimBlock * IPT keys held in registers; warp w owns
// tile elements [w * 32 * IPT, (w + 1) * 32 * IPT), its lane l the elements
// w * 32 * IPT + r * 32 + l (coalesced loads).  Ranks among equal digits
// follow element order: within a warp, round by round from
// __match_any_sync and the warp's own digit counters (warp-synchronous);
// across warps, from a prefix of the warps' counts per digit.  The tile is
// then rearranged by digit in shared memory and written out so that each
// digit's run lands on consecutive addresses (coalesced sectors instead of
// one sector per key).
template <int W, int IPT>
__global__ void __launch_bounds__(kPrimBlock) k_scatter(const uint32_t *d_n, const KeyW<W> *kin,
                                                        const uint32_t *vin, KeyW<W> *kout,
                                                        uint32_t *vout, int pass,
                                                        const uint32_t *offs) {
  constexpr int NW = kPrimBlock / 32, TILE = kPrimBlock * IPT;
  __shared__ uint32_t s_base[256];   // next global position per digit
  __shared__ uint32_t s_run[256];    // keys of the digit in the tile
  __shared__ uint32_t s_start[256];  // first tile position of the digit
  __shared__ uint32_t s_cnt[NW][256];  // per warp: count, then exclusive prefix
  __shared__ KeyW<W> s_key[TILE];
  __shared__ uint32_t s_val[TILE];
  __shared__ uint16_t s_dig[TILE];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const uint32_t lt = (1u << lane) - 1u;
  s_base[t] = offs[blockIdx.x * 256 + t];
  const uint32_t n = *d_n;
  uint32_t lo, hi;
  block_range(n, lo, hi);
  for (uint32_t r0 = lo; r0 < hi; r0 += TILE) {
    for (int w = 0; w < NW; w++) s_cnt[w][t] = 0;
    KeyW<W> k[IPT];
    uint32_t v[IPT], dg[IPT], rank[IPT];
    const uint32_t wbase = r0 + (uint32_t)warp * 32u * IPT + lane;
#pragma unroll
    for (int r = 0; r < IPT; r++) {
      const uint32_t i = wbase + 32u * r;
      dg[r] = 256;
      v[r] = 0;
      if (i < hi) {
        k[r] = kin[i];
        v[r] = vin[i];
        dg[r] = digit_of<W>(k[r], pass);
      }
    }
    __syncthreads();
    // ranks within the warp, in element order
#pragma unroll
    for (int r = 0; r < IPT; r++) {
      const uint32_t peers = __match_any_sync(0xffffffffu, dg[r]);
      const uint32_t c = dg[r] < 256 ? s_cnt[warp][dg[r]] : 0u;
      rank[r] = c + __popc(peers & lt);
      __syncwarp();
      if (dg[r] < 256 && (peers & lt) == 0) s_cnt[warp][dg[r]] = c + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    {  // per digit t: exclusive prefix over the warps, tile total
      uint32_t run = 0;
      for (int w = 0; w < NW; w++) {
        const uint32_t c = s_cnt[w][t];
        s_cnt[w][t] = run;
        run += c;
      }
      s_run[t] = run;
    }
    __syncthreads();
    // digit starts within the tile: exclusive scan of s_run (one warp)
    if (warp == 0) {
      uint32_t c[8], sum = 0;
#pragma unroll
      for (int q = 0; q < 8; q++) {
        c[q] = s_run[lane * 8 + q];
        sum += c[q];
      }
      uint32_t incl = sum;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      uint32_t run = incl - sum;
#pragma unroll
      for (int q = 0; q < 8; q++) {
        s_start[lane * 8 + q] = run;
        run += c[q];
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < IPT; r++) {
      const uint32_t p =
          dg[r] < 256 ? s_start[dg[r]] + s_cnt[warp][dg[r]] + rank[r] : (uint32_t)TILE;
      if (p < (uint32_t)TILE) {
        s_key[p] = k[r];
        s_val[p] = v[r];
        s_dig[p] = (uint16_t)dg[r];
      }
    }
    __syncthreads();
    const uint32_t n_tile = min((uint32_t)TILE, hi - r0);
    for (uint32_t p = t; p < n_tile; p += kPrimBlock) {
      const uint32_t d = s_dig[p] & 255u;
      const uint32_t pos = s_base[d] + (p - s_start[d]);
      if (pos < n) {
        kout[pos] = s_key[p];
        vout[pos] = s_val[p];
      }
    }
    __syncthreads();
    s_base[t] += s_run[t];
  }
}

__global__ void __launch_bounds__(kPrimBlock) k_scan_reduce(const uint32_t *d_n, const uint32_t *in,
                                                            uint32_t *partial) {
  __shared__ uint32_t sh[kPrimBlock / 32];
  uint32_t lo, hi;
  block_range(*d_n, lo, hi);
  uint32_t s = 0;
  for (uint32_t i = lo + threadIdx.x; i < hi; i += kPrimBlock) s += in[i];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kPrimBlock / 32; w++) t += sh[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kPrimBlock) k_scan_down(const uint32_t *d_n, const uint32_t *in,
                                                          uint32_t *out, const uint32_t *partial) {
  __shared__ uint32_t sh[kPrimBlock / 32];
  __shared__ uint32_t carry;
  uint32_t lo, hi;
  block_range(*d_n, lo, hi);
  if (threadIdx.x == 0) carry = partial[blockIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t r0 = lo; r0 < hi; r0 += kPrimBlock) {
    uint32_t i = r0 + threadIdx.x;
    uint32_t x = i < hi ? in[i] : 0;
    uint32_t incl = x;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) sh[warp] = incl;
    __syncthreads();
    uint32_t wbase = 0, tot = 0;
    for (int w = 0; w < kPrimBlock / 32; w++) {
      uint32_t c = sh[w];
      if (w < warp) wbase += c;
      tot += c;
    }
    if (i < hi) out[i] = carry + wbase + incl - x;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
}

}  // namespace

template <int W>
bool radix_sort(const uint32_t *d_n, KeyW<W> *keys, uint32_t *vals, KeyW<W> *keys2,
                uint32_t *vals2, int bits, uint32_t *hist, cudaStream_t s, uint64_t max_n,
                int first_pass) {
  int passes = (bits + 7) / 8;
  // blocks: about 8 tiles of 256 keys each for the largest possible count
  int G = (int)std::min<uint64_t>(kPrimGrid, std::max<uint64_t>(1, (max_n + 2047) / 2048));
  bool alt = false;
  for (int p = first_pass; p < passes; p++) {
    KeyW<W> *ki = alt ? keys2 : keys, *ko = alt ? keys : keys2;
    uint32_t *vi = alt ? vals2 : vals, *vo = alt ? vals : vals2;
    emrt::note_launch(), k_hist<W><<<G, kPrimBlock, 0, s>>>(d_n, ki, p, hist);
    emrt::note_launch(), k_digit_offsets<<<1, 1024, 0, s>>>(d_n, hist, G);
    emrt::note_launch(), k_scatter<W, (W == 4 ? 4 : 8)><<<G, kPrimBlock, 0, s>>>(d_n, ki, vi, ko, vo, p, hist);
    alt = !alt;
  }
  return alt;
}

template bool radix_sort<1>(const uint32_t *, KeyW<1> *, uint32_t *, KeyW<1> *, uint32_t *,
                            int, uint32_t *, cudaStream_t, uint64_t, int);
template bool radix_sort<2>(const uint32_t *, KeyW<2> *, uint32_t *, KeyW<2> *, uint32_t *,
                            int, uint32_t *, cudaStream_t, uint64_t, int);
template bool radix_sort<4>(const uint32_t *, KeyW<4> *, uint32_t *, KeyW<4> *, uint32_t *,
                            int, uint32_t *, cudaStream_t, uint64_t, int);

void exclusive_scan(const uint32_t *d_n, const uint32_t *in, uint32_t *out, uint32_t *d_total,
                    uint32_t *partial, cudaStream_t s) {
  emrt::note_launch(), k_scan_reduce<<<kPrimGrid, kPrimBlock, 0, s>>>(d_n, in, partial);
  emrt::note_launch(), k_scan_single<<<1, 1024, 0, s>>>(partial, kPrimGrid, d_total);
  emrt::note_launch(), k_scan_down<<<kPrimGrid, kPrimBlock, 0, s>>>(d_n, in, out, partial);
}

}  // namespace emrt
