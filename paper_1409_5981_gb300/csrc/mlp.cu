// Kernels of the learned local-expansion correction: a multilayer perceptron
// 432 -> 256 -> 256 -> 121 (GELU) with BF16 operands and FP32 accumulation on
// the tensor cores, its training (loss, backpropagation, Adam) and the data
// movement between the PMMM cell arrays and the network's row-major batches.
//
// GEMM: D[M x N] = A[M x K] . B[N x K]^T with A and B BF16 row-major (K
// contiguous).  A CTA of 128 threads owns a 128 x TN tile (TN = 64, 128, 256):
// K is staged 64 at a time into shared memory with 16-byte cp.async copies
// (zero-filled past K or N) in the no-swizzle K-major core-matrix layout, two
// stages deep; one thread issues the four K = 16 MMAs of a stage into the TMEM
// accumulator and commits them to the stage's mbarrier, which frees the stage
// for the copy two chunks ahead.  The epilogue reads the accumulator lane =
// row, 16 columns at a time, and applies bias, GELU or the GELU derivative.
#include <cuda_bf16.h>

#include "internal.cuh"
#include "tcgen05.cuh"

namespace pmmm {

namespace {

constexpr int G_THREADS = 128;
constexpr int G_KC = 64;                       // K per stage
constexpr uint32_t G_LBO = 128, G_SBO = 1024;  // 8 K-groups of 128 B per 8-row group
constexpr uint32_t G_A_BYTES = 128 * G_KC * 2;
constexpr long long G_WAIT_LIMIT = 1ll << 26;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_prime(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ void cp16(uint32_t saddr, const void* g, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(g), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ uint32_t chunk_off(int r, int g) {
  return (uint32_t)(r >> 3) * G_SBO + (uint32_t)g * G_LBO + (uint32_t)(r & 7) * 16;
}

template <int TN>
__global__ void __launch_bounds__(G_THREADS) gemm_tc_kernel(GemmArgs a) {
  constexpr uint32_t B_BYTES = TN * G_KC * 2;
  constexpr uint32_t STAGE = G_A_BYTES + B_BYTES;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * STAGE);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 2 * STAGE + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t m0 = (int64_t)blockIdx.x * 128;
  const int n0 = blockIdx.y * TN;
  const int nchunks = (a.K + G_KC - 1) / G_KC;
  const uint32_t sbase = tc::smem_u32(smem);

  if (tid == 0) {
    tc::bar_init(tc::smem_u32(&bars[0]), 1);
    tc::bar_init(tc::smem_u32(&bars[1]), 1);
    tc::fence_proxy_async();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, TN);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;

  auto load = [&](int ch, int st) {
    const int k0 = ch * G_KC;
    const uint32_t sa = sbase + st * STAGE, sb = sa + G_A_BYTES;
    for (int pi = tid; pi < 128 * 8; pi += G_THREADS) {
      const int r = pi >> 3, g = pi & 7, k = k0 + 8 * g;
      const bool ok = k < a.K;
      cp16(sa + chunk_off(r, g), ok ? (const void*)(a.A + (m0 + r) * a.lda + k) : (const void*)a.A, ok);
    }
    for (int pi = tid; pi < TN * 8; pi += G_THREADS) {
      const int r = pi >> 3, g = pi & 7, k = k0 + 8 * g;
      const bool ok = k < a.K && n0 + r < a.N;
      cp16(sb + chunk_off(r, g), ok ? (const void*)(a.B + (int64_t)(n0 + r) * a.ldb + k) : (const void*)a.B, ok);
    }
    cp_commit();
  };

  bool ok = true;
  load(0, 0);
  const uint32_t idesc = tc::idesc_bf16_m128(TN);
  for (int ch = 0; ch < nchunks; ++ch) {
    const int st = ch & 1;
    if (ch + 1 < nchunks) {
      // the other stage was read by the MMAs of chunk ch - 1
      if (ch >= 1 && !tc::bar_wait(tc::smem_u32(&bars[st ^ 1]), (uint32_t)(((ch - 1) >> 1) & 1), G_WAIT_LIMIT)) ok = false;
      load(ch + 1, st ^ 1);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t sa = sbase + st * STAGE, sb = sa + G_A_BYTES;
#pragma unroll
      for (int j = 0; j < G_KC / 16; ++j)
        tc::mma_bf16(tmem, tc::desc(sa + 256 * j, G_LBO, G_SBO), tc::desc(sb + 256 * j, G_LBO, G_SBO), idesc,
                     (ch | j) != 0);
      tc::commit(tc::smem_u32(&bars[st]));
    }
  }
  const int last = nchunks - 1;
  if (!__all_sync(0xffffffffu, tc::bar_wait(tc::smem_u32(&bars[last & 1]), (uint32_t)((last >> 1) & 1), G_WAIT_LIMIT)))
    ok = false;
  tc::fence_after();
  if (__all_sync(0xffffffffu, ok)) {
    const int64_t row = m0 + 32 * warp + lane;
    for (int cc = 0; cc < TN; cc += 16) {
      const int col = n0 + cc;
      if (col >= a.N) break;  // N is a multiple of 16: a column group is all in or all out
      float v[16];
      tc::ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cc, v);
      tc::wait_ld();
      if (a.bias) {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] += a.bias[col + j];
      }
      if (a.epi == GEMM_EPI_DGELU) {
        const float4* zp = reinterpret_cast<const float4*>(a.Zin + row * a.ldz + col);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 z = zp[q];
          v[4 * q] *= gelu_prime(z.x);
          v[4 * q + 1] *= gelu_prime(z.y);
          v[4 * q + 2] *= gelu_prime(z.z);
          v[4 * q + 3] *= gelu_prime(z.w);
        }
      }
      if (a.D32) {
        float4* dp = reinterpret_cast<float4*>(a.D32 + row * a.ldd + col);
#pragma unroll
        for (int q = 0; q < 4; ++q) dp[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
      if (a.D16) {
        uint32_t h[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float x0 = v[2 * q], x1 = v[2 * q + 1];
          if (a.epi == GEMM_EPI_GELU) {
            x0 = gelu(x0);
            x1 = gelu(x1);
          }
          const __nv_bfloat162 b = __floats2bfloat162_rn(x0, x1);
          h[q] = *reinterpret_cast<const uint32_t*>(&b);
        }
        uint4* hp = reinterpret_cast<uint4*>(a.D16 + row * a.ldd16 + col);
        hp[0] = make_uint4(h[0], h[1], h[2], h[3]);
        hp[1] = make_uint4(h[4], h[5], h[6], h[7]);
      }
    }
  } else if (tid == 0 && a.err) {
    set_err(a.err, ERRBIT_TIMEOUT);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, TN);
}

// out[c][r] = in[r][c] for a BF16 R x C matrix (row strides ld_in, ld_out)
__global__ void __launch_bounds__(256) transpose_bf16_kernel(const __nv_bfloat16* __restrict__ in, int64_t ld_in,
                                                             __nv_bfloat16* __restrict__ out, int64_t ld_out, int R,
                                                             int C) {
  __shared__ __nv_bfloat16 tile[32][34];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.y * 32;
  const int c0 = blockIdx.x * 32;
  for (int j = ty; j < 32; j += 8) {
    const int64_t r = r0 + j;
    const int c = c0 + tx;
    tile[j][tx] = (r < R && c < C) ? in[r * ld_in + c] : __float2bfloat16(0.f);
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int c = c0 + j;
    const int64_t r = r0 + tx;
    if (c < C && r < R) out[(int64_t)c * ld_out + r] = tile[tx][j];
  }
}

// out[c] = sum over rows of in[r][c] (FP32 in, FP64 sum in a fixed order)
__global__ void __launch_bounds__(256) colsum_kernel(const float* __restrict__ in, int64_t ld, int R, int C,
                                                     float* __restrict__ out) {
  __shared__ double sh[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + tx;
  double acc = 0.0;
  if (c < C)
    for (int r = ty; r < R; r += 8) acc += (double)in[(int64_t)r * ld + c];
  sh[ty][tx] = acc;
  __syncthreads();
  if (ty == 0 && c < C) {
    double t = 0.0;
    for (int j = 0; j < 8; ++j) t += sh[j][tx];
    out[c] = (float)t;
  }
}

// dO = 2 (O - T) / (rows * nout) on the first nout columns (0 beyond), FP32 and
// BF16; per-block partial sums of (O - T)^2 in FP64.
__global__ void __launch_bounds__(256) mse_grad_kernel(const float* __restrict__ O, const float* __restrict__ T,
                                                       int64_t rows, int ld, int nout, float* __restrict__ dO,
                                                       __nv_bfloat16* __restrict__ dO16, double* __restrict__ part) {
  __shared__ double sh[256];
  const double scale = 2.0 / ((double)rows * nout);
  double acc = 0.0;
  const int64_t total = rows * ld;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < total; i += (int64_t)gridDim.x * 256) {
    const int c = (int)(i % ld);
    float g = 0.f;
    if (c < nout) {
      const float d = O[i] - T[i];
      acc += (double)d * d;
      g = (float)(scale * d);
    }
    dO[i] = g;
    dO16[i] = __float2bfloat16(g);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void sum_partials_kernel(const double* __restrict__ part, int n, double scale, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += part[i];
    *out = t * scale;
  }
}

// Adam (Kingma & Ba) on the FP32 master parameters.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16(in[i]);
}

// Features of every cell: the 16 device-unit multipoles (p = 3) of the 27 cells
// (dz, dy, dx) in {-1, 0, 1}^3 around it, neighbour-major, each channel times
// in_scale[channel]; open boundaries give zeros outside the mesh.
__global__ void __launch_bounds__(256) gather_features_kernel(const float* __restrict__ M, int64_t K, int nx, int ny,
                                                              int nz, int periodic, const float* __restrict__ in_scale,
                                                              __nv_bfloat16* __restrict__ X, int64_t ldx) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= K * 27) return;
  const int64_t cell = t / 27;
  const int nb = (int)(t - cell * 27);
  const int ix = (int)(cell % nx), iy = (int)((cell / nx) % ny), iz = (int)(cell / ((int64_t)nx * ny));
  int jx = ix + nb % 3 - 1, jy = iy + (nb / 3) % 3 - 1, jz = iz + nb / 9 - 1;
  bool ok = true;
  if (jx < 0 || jx >= nx) { ok = ok && periodic; jx = (jx + nx) % nx; }
  if (jy < 0 || jy >= ny) { ok = ok && periodic; jy = (jy + ny) % ny; }
  if (jz < 0 || jz >= nz) { ok = ok && periodic; jz = (jz + nz) % nz; }
  const int64_t cj = jx + (int64_t)nx * (jy + (int64_t)ny * jz);
  uint32_t h[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float x0 = 0.f, x1 = 0.f;
    if (ok) {
      x0 = M[(int64_t)(2 * q) * K + cj] * in_scale[2 * q];
      x1 = M[(int64_t)(2 * q + 1) * K + cj] * in_scale[2 * q + 1];
    }
    const __nv_bfloat162 b = __floats2bfloat162_rn(x0, x1);
    h[q] = *reinterpret_cast<const uint32_t*>(&b);
  }
  uint4* o = reinterpret_cast<uint4*>(X + cell * ldx + nb * 16);
  o[0] = make_uint4(h[0], h[1], h[2], h[3]);
  o[1] = make_uint4(h[4], h[5], h[6], h[7]);
}

// Targets: T[cell][c] = (Lhi[c][cell] - (c < clow ? Llo[c][cell] : 0)) * out_scale[c] for
// c < chi, zero up to ldt.  Also FP64 sums of squares of the raw differences per channel.
__global__ void __launch_bounds__(256) build_targets_kernel(const float* __restrict__ Lhi, const float* __restrict__ Llo,
                                                            int64_t K, int chi, int clow,
                                                            const float* __restrict__ out_scale, float* __restrict__ T,
                                                            int ldt) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= K * ldt) return;
  const int64_t cell = t / ldt;
  const int c = (int)(t - cell * ldt);
  float v = 0.f;
  if (c < chi) v = (Lhi[(int64_t)c * K + cell] - (c < clow ? Llo[(int64_t)c * K + cell] : 0.f)) * out_scale[c];
  T[t] = v;
}

// Corrected locals for L2P at the high order: L[c][cell] = (c < clow ? Llo[c][cell] : 0) + O[cell][c] / out_scale[c].
__global__ void __launch_bounds__(256) combine_locals_kernel(const float* __restrict__ Llo, const float* __restrict__ O,
                                                             int ldo, int64_t K, int chi, int clow,
                                                             const float* __restrict__ out_scale,
                                                             float* __restrict__ L) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= K * chi) return;
  const int c = (int)(t / K);
  const int64_t cell = t - (int64_t)c * K;
  L[t] = (c < clow ? Llo[(int64_t)c * K + cell] : 0.f) + O[cell * ldo + c] / out_scale[c];
}

// FP64 sums of squares per channel of a channel-major FP32 array [C][K]
__global__ void __launch_bounds__(256) channel_sumsq_kernel(const float* __restrict__ X, int64_t K,
                                                            double* __restrict__ out) {
  __shared__ double sh[256];
  const int c = blockIdx.x;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < K; i += 256) {
    const double x = X[(int64_t)c * K + i];
    acc += x * x;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] += sh[0];
}

// same for the difference Lhi - Llo (channels c < clow) / Lhi (c >= clow)
__global__ void __launch_bounds__(256) diff_sumsq_kernel(const float* __restrict__ Lhi, const float* __restrict__ Llo,
                                                         int64_t K, int clow, double* __restrict__ out) {
  __shared__ double sh[256];
  const int c = blockIdx.x;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < K; i += 256) {
    const double x = (double)Lhi[(int64_t)c * K + i] - (c < clow ? (double)Llo[(int64_t)c * K + i] : 0.0);
    acc += x * x;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] += sh[0];
}

unsigned grid_for(int64_t n, int threads, int64_t cap = 1 << 20) {
  return (unsigned)std::min<int64_t>(cap, std::max<int64_t>(1, (n + threads - 1) / threads));
}

}  // namespace

cudaError_t launch_gemm_tc(const GemmArgs& a, cudaStream_t s, int* nl) {
  if (a.M <= 0 || a.N <= 0) return cudaSuccess;
  if (a.M % 128 || a.N % 16 || a.K % 16 || a.K <= 0 || a.lda % 8 || a.ldb % 8) return cudaErrorInvalidValue;
  if ((a.D32 && a.ldd % 4) || (a.D16 && a.ldd16 % 8) || (a.epi == GEMM_EPI_DGELU && (!a.Zin || a.ldz % 4)))
    return cudaErrorInvalidValue;
  const int TN = a.N > 128 ? 256 : (a.N > 64 ? 128 : 64);
  const size_t smem = 2 * ((size_t)G_A_BYTES + (size_t)TN * G_KC * 2) + 64;
  dim3 grid((unsigned)(a.M / 128), (unsigned)((a.N + TN - 1) / TN));
  cudaError_t e;
#define GEMM_LAUNCH(T)                                                                                   \
  e = cudaFuncSetAttribute(gemm_tc_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
  if (e != cudaSuccess) return e;                                                                       \
  gemm_tc_kernel<T><<<grid, G_THREADS, smem, s>>>(a)
  if (TN == 256) {
    GEMM_LAUNCH(256);
  } else if (TN == 128) {
    GEMM_LAUNCH(128);
  } else {
    GEMM_LAUNCH(64);
  }
#undef GEMM_LAUNCH
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_transpose_bf16(const void* in, int64_t ld_in, void* out, int64_t ld_out, int R, int C,
                                  cudaStream_t s, int* nl) {
  if (R <= 0 || C <= 0) return cudaSuccess;
  dim3 grid((unsigned)((C + 31) / 32), (unsigned)((R + 31) / 32));
  transpose_bf16_kernel<<<grid, 256, 0, s>>>((const __nv_bfloat16*)in, ld_in, (__nv_bfloat16*)out, ld_out, R, C);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_colsum(const float* in, int64_t ld, int R, int C, float* out, cudaStream_t s, int* nl) {
  colsum_kernel<<<(unsigned)((C + 31) / 32), 256, 0, s>>>(in, ld, R, C, out);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_mse_grad(const float* O, const float* T, int64_t rows, int ld, int nout, float* dO, void* dO16,
                            double* part, int nparts, double* loss, cudaStream_t s, int* nl) {
  mse_grad_kernel<<<(unsigned)nparts, 256, 0, s>>>(O, T, rows, ld, nout, dO, (__nv_bfloat16*)dO16, part);
  sum_partials_kernel<<<1, 32, 0, s>>>(part, nparts, 1.0 / ((double)rows * nout), loss);
  *nl += 2;
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, int64_t step, cudaStream_t s,
                        int* nl) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = (float)(1.0 - pow(0.9, (double)step)), c2 = (float)(1.0 - pow(0.999, (double)step));
  adam_kernel<<<grid_for(n, 256, 4096), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, 1e-8f, c1, c2);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* in, void* out, int64_t n, cudaStream_t s, int* nl) {
  to_bf16_kernel<<<grid_for(n, 256, 4096), 256, 0, s>>>(in, (__nv_bfloat16*)out, n);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_gather_features(const float* M, int64_t K, const int n[3], int periodic, const float* in_scale,
                                   void* X, int64_t ldx, cudaStream_t s, int* nl) {
  gather_features_kernel<<<grid_for(K * 27, 256, 1ll << 31), 256, 0, s>>>(M, K, n[0], n[1], n[2], periodic, in_scale,
                                                                         (__nv_bfloat16*)X, ldx);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_build_targets(const float* Lhi, const float* Llo, int64_t K, int chi, int clow,
                                 const float* out_scale, float* T, int ldt, cudaStream_t s, int* nl) {
  build_targets_kernel<<<grid_for(K * ldt, 256, 1ll << 31), 256, 0, s>>>(Lhi, Llo, K, chi, clow, out_scale, T, ldt);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_combine_locals(const float* Llo, const float* O, int ldo, int64_t K, int chi, int clow,
                                  const float* out_scale, float* L, cudaStream_t s, int* nl) {
  combine_locals_kernel<<<grid_for(K * chi, 256, 1ll << 31), 256, 0, s>>>(Llo, O, ldo, K, chi, clow, out_scale, L);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_channel_sumsq(const float* X, int C, int64_t K, double* out, cudaStream_t s, int* nl) {
  channel_sumsq_kernel<<<(unsigned)C, 256, 0, s>>>(X, K, out);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_diff_sumsq(const float* Lhi, const float* Llo, int C, int clow, int64_t K, double* out,
                              cudaStream_t s, int* nl) {
  diff_sumsq_kernel<<<(unsigned)C, 256, 0, s>>>(Lhi, Llo, K, clow, out);
  ++*nl;
  return cudaGetLastError();
}

}  // namespace pmmm
