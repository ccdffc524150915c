// Binning and stable counting sort of the particles by cell (Sec. 2.1: "for
// each cell, the set of particles inside is known ... in an O(N) procedure").
//
// Cell index, in FP64 with every operation rounded (no contraction):
//   t = x - lo;  if t is outside [0, len):
//     periodic: t = t - len * floor(t / len), and t -= len if t >= len
//     open: flag OUT_OF_BOX
//   i = floor(t * (n / len)) clamped to [0, n-1];  id = ix + nx (iy + ny iz)
// The sort is an LSD radix sort on the id (digits of <= 8 bits), stable in
// every pass, so the particles of a cell keep their input order.
#include "binning.cuh"
#include "internal.cuh"

namespace pmmm {

namespace {
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // 2048 keys per tile
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_CH = SCAN_THREADS * 4;  // entries per scan chunk

template <typename T>
__global__ void bin_kernel(const T* __restrict__ pos, const T* __restrict__ q, int64_t n, Geo g,
                           uint32_t* __restrict__ keys, T* __restrict__ rec, int* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) bin_record<T>(pos, q, i, g, 0u, keys, rec, err);
}

__global__ void radix_hist_kernel(const uint32_t* __restrict__ keys, int64_t n, int shift, int nbits,
                                  uint32_t* __restrict__ hist, int ntiles) {
  __shared__ uint32_t cnt[256];
  const int radix = 1 << nbits;
  for (int t = threadIdx.x; t < radix; t += RS_THREADS) cnt[t] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
  for (int k = 0; k < RS_ITEMS; ++k) {
    const int64_t i = base + k * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & (radix - 1)], 1u);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < radix; t += RS_THREADS) hist[(int64_t)t * ntiles + blockIdx.x] = cnt[t];
}

// Block-wide exclusive scan of SCAN_CH entries in place; writes the chunk total.
__global__ void scan_chunks_kernel(uint32_t* __restrict__ data, int64_t total, uint32_t* __restrict__ sums) {
  __shared__ uint32_t wsum[SCAN_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_CH + (int64_t)threadIdx.x * 4;
  uint32_t v[4];
  uint32_t local = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = (base + k < total) ? data[base + k] : 0u;
    local += v[k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = (lane < SCAN_THREADS / 32) ? wsum[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < SCAN_THREADS / 32) wsum[lane] = wi - w;  // exclusive warp offsets
    if (lane == 31) sums[blockIdx.x] = wi;
  }
  __syncthreads();
  uint32_t run = wsum[warp] + incl - local;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (base + k < total) data[base + k] = run;
    run += v[k];
  }
}

// Exclusive scan of the chunk totals (one block, sequential over groups of 1024).
__global__ void scan_top_kernel(uint32_t* __restrict__ sums, int nchunks) {
  __shared__ uint32_t wsum[SCAN_THREADS / 32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < nchunks; base += SCAN_THREADS) {
    const int i = base + threadIdx.x;
    const uint32_t v = (i < nchunks) ? sums[i] : 0u;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = wsum[lane];
      uint32_t wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
      }
      wsum[lane] = wi - w;
    }
    __syncthreads();
    const uint32_t c0 = carry;
    if (i < nchunks) sums[i] = c0 + wsum[warp] + incl - v;
    __syncthreads();
    if (threadIdx.x == SCAN_THREADS - 1) carry = c0 + wsum[warp] + incl;
    __syncthreads();
  }
}

// Stable scatter of one radix pass.  Warp w of a tile owns keys
// [w*256, (w+1)*256) of the tile, visited in 8 rounds of 32 in index order, so
// that ranks among equal digits follow the input order.  The tile is first
// grouped by digit in shared memory (stable), then written out position by
// position, so that keys of one digit leave as one contiguous run.
__global__ void radix_scatter_kernel(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                     uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n, int shift,
                                     int nbits, const uint32_t* __restrict__ hist, const uint32_t* __restrict__ chunks,
                                     int ntiles) {
  __shared__ uint32_t whist[RS_WARPS][256];
  __shared__ uint32_t gbase[256];
  __shared__ uint32_t tdo[256];  // first tile position of each digit
  __shared__ uint32_t wtot[RS_WARPS];
  __shared__ uint32_t sk[RS_TILE], sv[RS_TILE];
  const int radix = 1 << nbits;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < RS_WARPS * 256; t += RS_THREADS) (&whist[0][0])[t] = 0;
  __syncthreads();
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t tbase = (int64_t)blockIdx.x * RS_TILE;
  const int64_t wbase = tbase + (int64_t)warp * (32 * RS_ITEMS);
  const int tcount = (int)min((int64_t)RS_TILE, n - tbase);
  uint32_t key[RS_ITEMS], val[RS_ITEMS], rank[RS_ITEMS];
  int dig[RS_ITEMS];
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int64_t i = wbase + r * 32 + lane;
    const bool valid = i < n;
    const uint32_t k = valid ? kin[i] : 0u;
    const int d = valid ? (int)((k >> shift) & (uint32_t)(radix - 1)) : 0x10000;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t prev = valid ? whist[warp][d] : 0u;
    __syncwarp();
    const int leader = __ffs(peers) - 1;
    if (valid && lane == leader) whist[warp][d] = prev + __popc(peers);
    __syncwarp();
    rank[r] = prev + __popc(peers & lt);
    key[r] = k;
    val[r] = valid ? (vin ? vin[i] : (uint32_t)i) : 0u;
    dig[r] = d;
  }
  __syncthreads();
  // per digit: exclusive offsets of the warps, the tile total, the global base
  const int t = threadIdx.x;  // RS_THREADS == 256 >= radix: one digit per thread
  uint32_t total = 0;
  if (t < radix) {
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
      const uint32_t c = whist[w][t];
      whist[w][t] = total;
      total += c;
    }
    const int64_t idx = (int64_t)t * ntiles + blockIdx.x;
    gbase[t] = hist[idx] + chunks[idx / SCAN_CH];
  }
  // exclusive scan of the digit totals over the block -> tdo
  uint32_t incl = total;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wtot[warp] = incl;
  __syncthreads();
  uint32_t woff = 0;
  for (int w = 0; w < warp; ++w) woff += wtot[w];
  tdo[t] = woff + incl - total;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int d = dig[r];
    if (d < radix) {
      const uint32_t lp = tdo[d] + whist[warp][d] + rank[r];
      sk[lp] = key[r];
      sv[lp] = val[r];
    }
  }
  __syncthreads();
  for (int j = t; j < tcount; j += RS_THREADS) {
    const uint32_t k = sk[j];
    const int d = (int)((k >> shift) & (uint32_t)(radix - 1));
    const uint32_t dst = gbase[d] + ((uint32_t)j - tdo[d]);
    kout[dst] = k;
    vout[dst] = sv[j];
  }
}

__global__ void cell_bounds_kernel(const uint32_t* __restrict__ keys, int64_t n, int64_t K, int* __restrict__ cs) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s > n) return;
  const int64_t kprev = (s == 0) ? -1 : (int64_t)keys[s - 1];
  const int64_t k = (s == n) ? K : (int64_t)keys[s];
  for (int64_t c = kprev + 1; c <= k; ++c) cs[c] = (int)s;
}

__global__ void scan_add_kernel(uint32_t* __restrict__ data, int64_t n, const uint32_t* __restrict__ chunks) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) data[i] += chunks[i / SCAN_CH];
}

inline int grid1(int64_t n, int b) { return (int)((n + b - 1) / b); }
}  // namespace

int64_t scan_chunk_count(int64_t n) { return (n + SCAN_CH - 1) / SCAN_CH + 1; }

cudaError_t launch_exclusive_scan(uint32_t* data, int64_t n, uint32_t* chunks, cudaStream_t s, int* nl) {
  if (n <= 0) return cudaSuccess;
  const int nchunks = (int)((n + SCAN_CH - 1) / SCAN_CH);
  scan_chunks_kernel<<<nchunks, SCAN_THREADS, 0, s>>>(data, n, chunks);
  scan_top_kernel<<<1, SCAN_THREADS, 0, s>>>(chunks, nchunks);
  scan_add_kernel<<<grid1(n, 256), 256, 0, s>>>(data, n, chunks);
  *nl += 3;
  return cudaGetLastError();
}

int sort_tiles(int64_t n) { return (int)((n + RS_TILE - 1) / RS_TILE); }
size_t sort_hist_entries(int64_t n) { return (size_t)256 * (size_t)(sort_tiles(n) > 0 ? sort_tiles(n) : 1); }
size_t sort_chunk_entries(int64_t n) { return (sort_hist_entries(n) + SCAN_CH - 1) / SCAN_CH + 1; }

cudaError_t launch_bin(const void* pos, const void* q, bool fp64, int64_t n, const Geo& g, uint32_t* keys, void* rec,
                       int* err, cudaStream_t s, int* nl) {
  if (n <= 0) return cudaSuccess;
  if (fp64)
    bin_kernel<double><<<grid1(n, 256), 256, 0, s>>>((const double*)pos, (const double*)q, n, g, keys,
                                                     (double*)rec, err);
  else
    bin_kernel<float><<<grid1(n, 256), 256, 0, s>>>((const float*)pos, (const float*)q, n, g, keys, (float*)rec,
                                                    err);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_radix_sort(SortWork& w, int64_t n, int key_bits, uint32_t** keys_out, uint32_t** vals_out,
                              cudaStream_t s, int* nl) {
  uint32_t *ki = w.keys0, *ko = w.keys1, *vi = nullptr, *vo = w.vals1;
  if (n <= 0) {
    *keys_out = w.keys0;
    *vals_out = w.vals0;
    return cudaSuccess;
  }
  const int ntiles = sort_tiles(n);
  const int64_t total = (int64_t)256 * ntiles;
  const int nchunks = (int)((total + SCAN_CH - 1) / SCAN_CH);
  int passes = (key_bits + 7) / 8;
  if (passes == 0) {
    // a single cell: the identity permutation is the stable order
    passes = 1;
    key_bits = 1;
  }
  const int per = (key_bits + passes - 1) / passes;
  int shift = 0;
  for (int ps = 0; ps < passes; ++ps) {
    const int nb = (shift + per <= key_bits) ? per : key_bits - shift;
    radix_hist_kernel<<<ntiles, RS_THREADS, 0, s>>>(ki, n, shift, nb, w.hist, ntiles);
    scan_chunks_kernel<<<nchunks, SCAN_THREADS, 0, s>>>(w.hist, (int64_t)(1 << nb) * ntiles, w.chunks);
    scan_top_kernel<<<1, SCAN_THREADS, 0, s>>>(w.chunks, nchunks);
    radix_scatter_kernel<<<ntiles, RS_THREADS, 0, s>>>(ki, vi, ko, vo, n, shift, nb, w.hist, w.chunks, ntiles);
    *nl += 4;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    shift += nb;
    // ping-pong: keys0 <-> keys1; the first pass reads implicit indices and
    // writes vals1, later passes alternate vals1 <-> vals0
    uint32_t* t = ki;
    ki = ko;
    ko = t;
    if (vi == nullptr) {
      vi = vo;
      vo = w.vals0;
    } else {
      uint32_t* tv = vi;
      vi = vo;
      vo = tv;
    }
  }
  *keys_out = ki;
  *vals_out = vi;
  return cudaSuccess;
}

cudaError_t launch_cell_bounds(const uint32_t* keys, int64_t n, int64_t K, int* cs, cudaStream_t s, int* nl) {
  cell_bounds_kernel<<<grid1(n + 1, 256), 256, 0, s>>>(keys, n, K, cs);
  ++*nl;
  return cudaGetLastError();
}

}  // namespace pmmm
