// Batched M2L on the 5th-generation tensor cores (tcgen05), split-BF16 operands
// with FP32 accumulation in tensor memory.
//
// Per wavevector k, the M2L of all systems (Sec. 2.1, real-matrix form of
// App. A.8) is the complex product L~ = A~ M~ with A~ (C x C) assembled from the
// kernel spectra and M~ (C x B).  Written as one real product with interleaved
// rows,
//   [Re L_c ; Im L_c] (row 2c, 2c+1) = [[Re A_c, -Im A_c], [Im A_c, Re A_c]] . [Re M ; Im M],
// it is a D[128 x N] = W[128 x 128] X[128 x N] GEMM with C padded to 64 channels
// (p <= 7).  Each FP32 operand x is split into x_hi = bf16(x) and
// x_lo = bf16(x - x_hi); D accumulates W_hi X_hi + W_hi X_lo + W_lo X_hi (the
// lo-lo term, below 2^-18 relative, is dropped), so every product carries a
// relative error of at most about 3 * 2^-18.
//
// Spectra are wavevector-major ([k][c][system]), so each wavevector's M~ and L~
// are one contiguous block.  One CTA of 256 threads owns a contiguous range of wavevectors and a tile of up
// to 64 systems.  Per wavevector all threads build W and X in shared memory (two
// buffers), one thread issues the 24 MMAs (M = 128, N = 64 or less, K = 16) into
// one of two TMEM accumulators and commits them to an mbarrier, and while they
// run the threads drain the previous accumulator (tcgen05.ld) to global memory.
// Shared-memory operands use the no-swizzle K-major layout of core matrices
// (8 rows x 16 bytes): element (r, k) at (r/8)*SBO + (k/8)*LBO + (r%8)*16 + (k%8)*2
// with LBO = 128 B and SBO = 2048 B.  Every mbarrier wait is bounded; on a
// timeout the kernel sets the plan's error flag, releases its tensor memory and
// returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "m2l_table.cuh"
#include "tcgen05.cuh"

namespace pmmm {

namespace {

constexpr int TC_THREADS = 512;  // 16 warps: the operand assembly is latency bound
constexpr int TC_CH = 64;                             // channels after padding (p <= 7)
constexpr int TC_K = 2 * TC_CH;                       // GEMM K: Re and Im parts of M
constexpr int TC_NMAX = 64;                           // largest system tile (GEMM N)
constexpr uint32_t TC_LBO = 128;                      // next core matrix along K
constexpr uint32_t TC_SBO = (TC_K / 8) * 128;         // next 8-row group: 2048 B
constexpr uint32_t TC_A_BYTES = 128 * TC_K * 2;       // one split of W: 32 KB
constexpr uint32_t TC_GK_BYTES = 2 * 2048;            // (2p+1)^2 <= 225 complex, two wavevectors
constexpr int TC_TAB_ROW = TC_CH + 4;                 // table row stride (words): 17 chunks of 16 B
constexpr uint32_t TC_TAB_BYTES = TC_CH * TC_TAB_ROW * 4;  // packed entry table, 17 KB
// per system tile NT (32 or 64): X splits, stage, shared-memory offsets, TMEM columns
template <int NT>
struct TcTile {
  static constexpr uint32_t B_BYTES = NT * TC_K * 2;                   // one split of X
  static constexpr uint32_t STAGE = 2 * TC_A_BYTES + 2 * B_BYTES;
  static constexpr uint32_t OFF_GK = 2 * STAGE;
  static constexpr uint32_t OFF_TAB = OFF_GK + TC_GK_BYTES;
  static constexpr uint32_t OFF_BAR = OFF_TAB + TC_TAB_BYTES;
  static constexpr uint32_t SMEM = OFF_BAR + 64;
  static constexpr uint32_t TMEM_COLS = 2 * NT;                         // two accumulators
};
constexpr long long TC_WAIT_LIMIT = 1ll << 26;        // mbarrier polls before giving up

using tc::smem_u32;

__device__ __forceinline__ uint64_t make_desc(uint32_t addr) { return tc::desc(addr, TC_LBO, TC_SBO); }
__device__ __forceinline__ uint32_t make_idesc(int n) { return tc::idesc_bf16_m128(n); }
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
  tc::mma_bf16(d, a, b, idesc, acc);
}
__device__ __forceinline__ void mma_commit(uint32_t bar) { tc::commit(bar); }
__device__ __forceinline__ void fence_after() { tc::fence_after(); }
__device__ __forceinline__ void fence_before() { tc::fence_before(); }
__device__ __forceinline__ void fence_proxy_async() { tc::fence_proxy_async(); }
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) { return tc::bar_wait(bar, parity, TC_WAIT_LIMIT); }
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) { tc::ld16(taddr, v); }
__device__ __forceinline__ void tmem_wait_ld() { tc::wait_ld(); }

// hi / lo BF16 split of 8 values, packed in K order (element j at the lower address).
__device__ __forceinline__ void split8(const float* x, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const __nv_bfloat162 bh = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
    const float r0 = x[2 * j] - __low2float(bh), r1 = x[2 * j + 1] - __high2float(bh);
    const __nv_bfloat162 bl = __floats2bfloat162_rn(r0, r1);
    h[j] = *reinterpret_cast<const uint32_t*>(&bh);
    l[j] = *reinterpret_cast<const uint32_t*>(&bl);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ uint4 neg_bf16(uint4 v) {
  return make_uint4(v.x ^ 0x80008000u, v.y ^ 0x80008000u, v.z ^ 0x80008000u, v.w ^ 0x80008000u);
}

// byte offset of the 16-byte chunk (row r, K-group g) in one operand
__device__ __forceinline__ uint32_t chunk_off(int r, int g) {
  return (uint32_t)(r >> 3) * TC_SBO + (uint32_t)g * TC_LBO + (uint32_t)(r & 7) * 16;
}

__device__ __forceinline__ void cp8(uint32_t saddr, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(saddr), "l"(g) : "memory");
}

// Entry table packing: i1 | (s1 + 1) << 10 | i2 << 12 | (s2 + 1) << 22
template <int NT>
__global__ void __launch_bounds__(TC_THREADS, 1)
    m2l_tc_kernel(const float2* __restrict__ Mt, const float2* __restrict__ Gt, float2* __restrict__ Lt,
                  const uint32_t* __restrict__ tab_g, int C, int CG, int B, int64_t Kh, int64_t kchunk,
                  int* __restrict__ err) {
  using Tl = TcTile<NT>;
  extern __shared__ __align__(1024) unsigned char smem[];
  float2* gkb = reinterpret_cast<float2*>(smem + Tl::OFF_GK);  // [2][256]: kernel spectra of k and k + 1
  uint32_t* tab = reinterpret_cast<uint32_t*>(smem + Tl::OFF_TAB);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Tl::OFF_BAR);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + Tl::OFF_BAR + 16);
  int* abort_flag = reinterpret_cast<int*>(smem + Tl::OFF_BAR + 20);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b0 = blockIdx.y * NT;
  const int nb = min(NT, B - b0);
  const int nmma = (nb + 15) & ~15;  // GEMM N: systems padded to a multiple of 16
  const int64_t kbeg = (int64_t)blockIdx.x * kchunk, kend = min(Kh, kbeg + kchunk);

  for (int i = tid; i < TC_CH * TC_CH; i += TC_THREADS) tab[(i / TC_CH) * TC_TAB_ROW + i % TC_CH] = tab_g[i];
  // kernel spectra of the first wavevector (asynchronous copies, 8 bytes each)
  auto fetch_gk = [&](int64_t kk, int slot) {
    if (kk < kend)
      for (int s = tid; s < CG; s += TC_THREADS) cp8(smem_u32(gkb + 256 * slot + s), Gt + (int64_t)s * Kh + kk);
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  fetch_gk(kbeg, 0);
  if (tid == 0) {
    tc::bar_init(smem_u32(&bars[0]), 1);
    tc::bar_init(smem_u32(&bars[1]), 1);
    *abort_flag = 0;
    fence_proxy_async();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, Tl::TMEM_COLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = make_idesc(nmma);
  const uint32_t sbase = smem_u32(smem);

  // drains accumulator `buf` (wavevector k) to Lt: warp w reads TMEM lanes 32 (w % 4) ...
  // (rows: Re / Im of channel row / 2) and columns 32 (w / 4) ... of the tile
  auto drain = [&](int buf, int64_t k, uint32_t parity) -> bool {
    // warp-uniform outcome: the TMEM loads below are .sync.aligned
    if (!__all_sync(0xffffffffu, bar_wait(smem_u32(&bars[buf]), parity))) return false;
    fence_after();
    // warp w reads TMEM lanes 32 (w % 4) ... and the 16 columns 16 (w / 4) ... (NT / 16 groups)
    const int cg = warp >> 2;
    if (cg >= NT / 16) {
      fence_before();
      return true;
    }
    const int row = 32 * (warp & 3) + lane;
    const int col0 = 16 * cg;
    float v[16];
    const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(buf * NT + col0);
    tmem_ld16(taddr, v);
    tmem_wait_ld();
    const int c = row >> 1;
    const bool odd = lane & 1;
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const float a = v[2 * jj], b = v[2 * jj + 1];
      const float recv = __shfl_xor_sync(0xffffffffu, odd ? a : b, 1);
      const int n = col0 + 2 * jj + (odd ? 1 : 0);
      if (c < C && n < nb) Lt[(k * C + c) * B + b0 + n] = odd ? make_float2(recv, b) : make_float2(a, recv);
    }
    fence_before();
    return true;
  };

  int it = 0;
  int64_t kprev = -1;
  bool ok = true;
  for (int64_t k = kbeg; k < kend; ++k, ++it) {
    const int buf = it & 1;
    unsigned char* st = smem + buf * Tl::STAGE;
    // this wavevector's kernel spectra were fetched one iteration ahead; start the next fetch
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    const float2* gk = gkb + 256 * (it & 1);
    fetch_gk(k + 1, (it + 1) & 1);
    // X loads first (their latency is covered by the W assembly below)
    float2 xm[(NT * 8 + TC_THREADS - 1) / TC_THREADS][8];
#pragma unroll
    for (int q = 0; q < (NT * 8 + TC_THREADS - 1) / TC_THREADS; ++q) {
      const int u = tid + q * TC_THREADS;
      const int n = (u & 7) + 8 * (u >> 6), cg = (u >> 3) & 7;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int ci = cg * 8 + j;
        xm[q][j] = make_float2(0.f, 0.f);
        if (u < NT * 8 && n < nb && ci < C) xm[q][j] = __ldg(Mt + (k * C + ci) * B + b0 + n);
      }
    }
    // W: unit (output channel co, K-group kg of 8 input channels) -> rows 2co, 2co+1; eight
    // consecutive threads take eight consecutive channels, whose padded table rows start on
    // different banks
    for (int u = tid; u < TC_CH * 8; u += TC_THREADS) {
      const int co = (u & 7) + 8 * (u >> 6), kg = (u >> 3) & 7;
      float ar[8], ai[8];
      uint32_t tv[8];
      *reinterpret_cast<uint4*>(tv) = *reinterpret_cast<const uint4*>(tab + co * TC_TAB_ROW + kg * 8);
      *reinterpret_cast<uint4*>(tv + 4) = *reinterpret_cast<const uint4*>(tab + co * TC_TAB_ROW + kg * 8 + 4);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint32_t t = tv[j];
        const float s1 = (float)((int)((t >> 10) & 3u) - 1), s2 = (float)((int)((t >> 22) & 3u) - 1);
        const float2 g1 = gk[t & 1023u], g2 = gk[(t >> 12) & 1023u];
        ar[j] = s1 * g1.x + s2 * g2.x;
        ai[j] = s1 * g1.y + s2 * g2.y;
      }
      uint4 rh, rl, ih, il;
      split8(ar, rh, rl);
      split8(ai, ih, il);
      unsigned char* Ah = st;
      unsigned char* Al = st + TC_A_BYTES;
      *reinterpret_cast<uint4*>(Ah + chunk_off(2 * co, kg)) = rh;
      *reinterpret_cast<uint4*>(Al + chunk_off(2 * co, kg)) = rl;
      *reinterpret_cast<uint4*>(Ah + chunk_off(2 * co, 8 + kg)) = neg_bf16(ih);
      *reinterpret_cast<uint4*>(Al + chunk_off(2 * co, 8 + kg)) = neg_bf16(il);
      *reinterpret_cast<uint4*>(Ah + chunk_off(2 * co + 1, kg)) = ih;
      *reinterpret_cast<uint4*>(Al + chunk_off(2 * co + 1, kg)) = il;
      *reinterpret_cast<uint4*>(Ah + chunk_off(2 * co + 1, 8 + kg)) = rh;
      *reinterpret_cast<uint4*>(Al + chunk_off(2 * co + 1, 8 + kg)) = rl;
    }
    // X: unit (system n, K-group cg of 8 channels) -> row n, K-groups cg (Re) and 8 + cg (Im)
#pragma unroll
    for (int q = 0; q < (NT * 8 + TC_THREADS - 1) / TC_THREADS; ++q) {
      const int u = tid + q * TC_THREADS;
      if (u >= NT * 8) break;
      const int n = (u & 7) + 8 * (u >> 6), cg = (u >> 3) & 7;
      float xr[8], xi[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        xr[j] = xm[q][j].x;
        xi[j] = xm[q][j].y;
      }
      uint4 rh, rl, ih, il;
      split8(xr, rh, rl);
      split8(xi, ih, il);
      unsigned char* Xh = st + 2 * TC_A_BYTES;
      unsigned char* Xl = Xh + Tl::B_BYTES;
      *reinterpret_cast<uint4*>(Xh + chunk_off(n, cg)) = rh;
      *reinterpret_cast<uint4*>(Xl + chunk_off(n, cg)) = rl;
      *reinterpret_cast<uint4*>(Xh + chunk_off(n, 8 + cg)) = ih;
      *reinterpret_cast<uint4*>(Xl + chunk_off(n, 8 + cg)) = il;
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      const uint32_t a_h = sbase + buf * Tl::STAGE, a_l = a_h + TC_A_BYTES;
      const uint32_t x_h = a_h + 2 * TC_A_BYTES, x_l = x_h + Tl::B_BYTES;
      const uint32_t d = tmem + (uint32_t)(buf * NT);
      const uint32_t As[3] = {a_h, a_h, a_l}, Xs[3] = {x_h, x_l, x_h};
#pragma unroll
      for (int sp = 0; sp < 3; ++sp)
#pragma unroll
        for (int j = 0; j < TC_K / 16; ++j)
          mma_bf16(d, make_desc(As[sp] + 256 * j), make_desc(Xs[sp] + 256 * j), idesc, (sp | j) != 0);
      mma_commit(smem_u32(&bars[buf]));
    }
    // the previous wavevector's accumulator, while these MMAs run
    if (kprev >= 0) {
      if (!drain(buf ^ 1, kprev, (uint32_t)(((it - 1) >> 1) & 1))) atomicExch(abort_flag, 1);
    }
    kprev = k;
    __syncthreads();
    if (*abort_flag) {
      ok = false;
      break;
    }
  }
  if (ok && kprev >= 0) {
    if (!drain((it - 1) & 1, kprev, (uint32_t)(((it - 1) >> 1) & 1))) atomicExch(abort_flag, 1);
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  if (*abort_flag) {
    if (tid == 0) set_err(err, ERRBIT_TIMEOUT);
    // give MMAs still in flight a bounded time to finish before the memory is released
    if (it >= 1) bar_wait(smem_u32(&bars[(it - 1) & 1]), (uint32_t)(((it - 1) >> 1) & 1));
  }
  fence_after();
  if (warp == 0) tc::tmem_free(tmem, Tl::TMEM_COLS);
}

}  // namespace

bool m2l_tc_supported(int p) { return p >= 0 && p <= 7; }

// Packed entry table of the real-matrix M2L, padded to 64 x 64 channels.
std::vector<uint32_t> build_m2l_table_tc(int p) {
  const int C = (p + 1) * (p + 1);
  std::vector<M2LEntry> t = build_m2l_table(p);
  std::vector<uint32_t> out((size_t)TC_CH * TC_CH, (1u << 10) | (1u << 22));  // both signs 0
  for (int co = 0; co < C; ++co)
    for (int ci = 0; ci < C; ++ci) {
      const M2LEntry& e = t[(size_t)co * C + ci];
      out[(size_t)co * TC_CH + ci] = (uint32_t)e.i1 | ((uint32_t)(e.s1 + 1) << 10) | ((uint32_t)e.i2 << 12) |
                                     ((uint32_t)(e.s2 + 1) << 22);
    }
  return out;
}

namespace {
template <int NT>
cudaError_t m2l_tc_run(const void* Mt, const void* Gt, void* Lt, const uint32_t* tab, int p, int B, int64_t Kh,
                       int num_sms, int* err, cudaStream_t s) {
  const int C = (p + 1) * (p + 1), CG = (2 * p + 1) * (2 * p + 1);
  const int ntiles = (B + NT - 1) / NT;
  const int per_tile = (int)std::max<int64_t>(1, std::min<int64_t>(Kh, (num_sms + ntiles - 1) / ntiles));
  const int64_t kchunk = (Kh + per_tile - 1) / per_tile;
  const unsigned gx = (unsigned)((Kh + kchunk - 1) / kchunk);
  const uint32_t smem = TcTile<NT>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(m2l_tc_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(gx, (unsigned)ntiles);
  m2l_tc_kernel<NT><<<grid, TC_THREADS, smem, s>>>((const float2*)Mt, (const float2*)Gt, (float2*)Lt, tab, C, CG, B,
                                                   Kh, kchunk, err);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_m2l_tc(const void* Mt, const void* Gt, void* Lt, const uint32_t* tab, int p, int B, int64_t Kh,
                          int num_sms, int tile, int* err, cudaStream_t s, int* nl) {
  if (!m2l_tc_supported(p) || B < 1) return cudaErrorInvalidValue;
  ++*nl;
  if (tile == 32) return m2l_tc_run<32>(Mt, Gt, Lt, tab, p, B, Kh, num_sms, err, s);
  return m2l_tc_run<64>(Mt, Gt, Lt, tab, p, B, Kh, num_sms, err, s);
}

}  // namespace pmmm

namespace pmmm {
namespace {
// One thread waits on an mbarrier that expects an arrival nobody makes, with the
// bounded wait of the tensor-core kernels; the timeout raises the error flag.
__global__ void wait_timeout_kernel(long long polls, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  tc::bar_init(tc::smem_u32(&bar), 1);
  if (!tc::bar_wait(tc::smem_u32(&bar), 0, polls)) set_err(err, ERRBIT_TIMEOUT);
}
}  // namespace
}  // namespace pmmm

extern "C" int pmmm_selftest_wait_timeout(void* cuda_stream, int64_t polls) {
  using namespace pmmm;
  if (polls < 1 || polls > (int64_t)1 << 24) return PMMM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int* err = nullptr;
  cudaError_t e = cudaMalloc(&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    wait_timeout_kernel<<<1, 32, 0, s>>>(polls, err);
    e = cudaGetLastError();
  }
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (err) cudaFree(err);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? PMMM_ERR_OOM : PMMM_ERR_CUDA;
  return (h & ERRBIT_TIMEOUT) ? PMMM_ERR_TIMEOUT : PMMM_OK;
}
