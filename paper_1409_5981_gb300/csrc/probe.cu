// Peak probes (measurement infrastructure, not part of the method): the FP32 and
// FP64 FMA rates of the GPU this library runs on, measured by kernels of
// independent FMA chains on every SM and timed with CUDA events.  They give the
// arithmetic rooflines of the ALU-bound kernels (near field, M2L) a measured
// denominator instead of a product of unit counts and clocks.
#include "internal.cuh"

namespace pmmm {

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;   // independent accumulators per thread
constexpr int PROBE_UNROLL = 8;   // chain steps per loop trip

// x <- x * a + b on PROBE_CHAINS independent chains; the result is stored only
// when it equals a value it cannot reach (x stays finite and near 1), so the
// chains are live but the store never happens.
__global__ void __launch_bounds__(PROBE_THREADS) fma32_probe_kernel(float* out, int iters, float a, float b) {
  float x[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = 1.0f + 1e-3f * (float)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
      for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
  if (s == -1.0f) out[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
}

__device__ __forceinline__ unsigned long long fma_x2(unsigned long long x, unsigned long long a,
                                                     unsigned long long b) {
  unsigned long long d;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(x), "l"(a), "l"(b));
  return d;
}

__global__ void __launch_bounds__(PROBE_THREADS) fma32x2_probe_kernel(float* out, int iters, float a, float b) {
  unsigned long long x[PROBE_CHAINS], av, bv;
  asm("mov.b64 %0, {%1, %2};" : "=l"(av) : "f"(a), "f"(a));
  asm("mov.b64 %0, {%1, %2};" : "=l"(bv) : "f"(b), "f"(b));
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) {
    const float v0 = 1.0f + 1e-3f * (float)(threadIdx.x + c), v1 = v0 + 0.5f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(v0), "f"(v1));
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
      for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fma_x2(x[c], av, bv);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
    s += lo + hi;
  }
  if (s == -1.0f) out[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) fma64_probe_kernel(double* out, int iters, double a, double b) {
  double x[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = 1.0 + 1e-3 * (double)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
      for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
  if (s == -1.0) out[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
}

}  // namespace

}  // namespace pmmm

using namespace pmmm;

extern "C" int pmmm_probe_peak(int what, void* cuda_stream, double* flops_per_s) {
  if (!flops_per_s || what < PMMM_PROBE_FP32_FMA || what > PMMM_PROBE_FP64_FMA) return PMMM_ERR_INVALID_ARG;
  *flops_per_s = 0.0;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return PMMM_ERR_CUDA;
  // eight resident blocks of 256 threads per SM: 64 warps, every scheduler full
  const int blocks = 8 * sms;
  const int iters = what == PMMM_PROBE_FP64_FMA ? 256 : 4096;
  void* out = nullptr;
  e = cudaMalloc(&out, sizeof(double) * (size_t)blocks * PROBE_THREADS);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? PMMM_ERR_OOM : PMMM_ERR_CUDA;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  float best = 0.f;
  for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {  // the first launch is a warm-up
    e = cudaEventRecord(t0, s);
    if (what == PMMM_PROBE_FP32_FMA)
      fma32_probe_kernel<<<blocks, PROBE_THREADS, 0, s>>>((float*)out, iters, 0.999999f, 1e-7f);
    else if (what == PMMM_PROBE_FP32X2_FMA)
      fma32x2_probe_kernel<<<blocks, PROBE_THREADS, 0, s>>>((float*)out, iters, 0.999999f, 1e-7f);
    else
      fma64_probe_kernel<<<blocks, PROBE_THREADS, 0, s>>>((double*)out, iters, 0.999999, 1e-7);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(t1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(out);
  if (e != cudaSuccess || best <= 0.f) return PMMM_ERR_CUDA;
  const double lanes = what == PMMM_PROBE_FP32X2_FMA ? 2.0 : 1.0;
  const double fmas = (double)blocks * PROBE_THREADS * iters * PROBE_UNROLL * PROBE_CHAINS * lanes;
  *flops_per_s = 2.0 * fmas / (best * 1e-3);
  return PMMM_OK;
}
