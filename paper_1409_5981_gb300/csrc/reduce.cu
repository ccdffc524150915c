// FP64 global reductions: the periodic correction terms of App. B.3 and the
// energy / net force.  Both are two-level tree reductions in one launch with a
// fixed assignment of cells to threads and of block partials to the final sum,
// so the results do not depend on scheduling.
#include "internal.cuh"

namespace pmmm {

namespace {

constexpr int RD_THREADS = 256;
constexpr int RD_BLOCKS = 256;
constexpr double kPi = 3.14159265358979323846;

template <int NQ>
__device__ void reduce_final(const double* __restrict__ partial, int nb, double* out) {
  __shared__ double sh[NQ][RD_THREADS];
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  for (int b = threadIdx.x; b < nb; b += RD_THREADS)
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] += __ldcg(partial + b * NQ + q);
#pragma unroll
  for (int q = 0; q < NQ; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = RD_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < NQ; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < NQ) out[threadIdx.x] = sh[threadIdx.x][0];
  __syncthreads();
}

// One launch for both levels of the tree: every block writes its NQ partial
// sums, and the block that finishes last (atomic ticket) sums all partials in
// block order into tot and re-arms the ticket.  Returns true in that block.
template <int NQ>
__device__ bool reduce_ticketed(const double* __restrict__ src, int64_t K, int64_t qstride, int64_t istride,
                                double* __restrict__ partial, unsigned int* __restrict__ ticket, double* tot) {
  __shared__ double sh[NQ][RD_THREADS];
  __shared__ bool last;
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  const int64_t per = (K + gridDim.x - 1) / gridDim.x;
  const int64_t beg = (int64_t)blockIdx.x * per, end = min(K, beg + per);
  for (int64_t i = beg + threadIdx.x; i < end; i += RD_THREADS)
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] += src[q * qstride + i * istride];
#pragma unroll
  for (int q = 0; q < NQ; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = RD_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < NQ; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < NQ) partial[blockIdx.x * NQ + threadIdx.x] = sh[threadIdx.x][0];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return false;
  __threadfence();
  reduce_final<NQ>(partial, gridDim.x, tot);
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// corr[0] = 2pi/(3V) sum q |r_rel|^2           (potential constant, App. B.3)
// corr[1..3] = -4pi/(3V) sum q r_rel           (dipole term of Eq. phicorr)
// corr[4] = 2pi/(3V) Q                         (charged-system factor)
// doubles 5..7 = FP32 copies of corr[0..4]
// corr[8..12] = Q, sum q u (3), sum q |u|^2 in units of hs
__global__ void __launch_bounds__(RD_THREADS) corrections_fused_kernel(const double* __restrict__ cellsum, int64_t K,
                                                                       double hs, double V,
                                                                       double* __restrict__ partial,
                                                                       unsigned int* __restrict__ ticket,
                                                                       double* __restrict__ corr) {
  __shared__ double tot[5];
  if (!reduce_ticketed<5>(cellsum, K, K, 1, partial, ticket, tot)) return;
  if (threadIdx.x == 0) {
    const double f = 2.0 * kPi / (3.0 * V);
    const double Q = tot[0];
    corr[0] = f * tot[4] * hs * hs;
    corr[1] = -2.0 * f * tot[1] * hs;
    corr[2] = -2.0 * f * tot[2] * hs;
    corr[3] = -2.0 * f * tot[3] * hs;
    corr[4] = f * Q;
    corr_store_f32(corr);
    for (int q = 0; q < 5; ++q) corr[8 + q] = tot[q];
  }
}

__global__ void __launch_bounds__(RD_THREADS) energy_fused_kernel(const double* __restrict__ epart, int64_t count,
                                                                  double* __restrict__ partial,
                                                                  unsigned int* __restrict__ ticket,
                                                                  double* __restrict__ energy) {
  __shared__ double tot[4];
  if (!reduce_ticketed<4>(epart, count, 1, 4, partial, ticket, tot)) return;
  if (threadIdx.x < 4) energy[threadIdx.x] = tot[threadIdx.x];
}

// channel c = sidx(l, m) of X (device units) times hs^(sh * l + off) -> FP64 out
template <typename T>
__global__ void to_physical_kernel(const T* __restrict__ X, double* __restrict__ out, int p, int64_t K, double hs,
                                   int mode) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int C = (p + 1) * (p + 1);
  if (i >= (int64_t)C * K) return;
  const int c = (int)(i / K);
  int l = 0;
  while ((l + 1) * (l + 1) <= c) ++l;
  // mode 0: multipoles M = M' hs^l ; mode 1: locals L = L' / hs^(l+1)
  const double f = mode == 0 ? pow(hs, (double)l) : pow(hs, -(double)(l + 1));
  out[i] = (double)X[i] * f;
}

}  // namespace

cudaError_t launch_corrections(const double* cellq, const double* celld, int64_t K, double hs, double V,
                               double* partial, unsigned int* ticket, double* corr, cudaStream_t s, int* nl) {
  // quantity 0 = cellq, quantities 1..4 = celld[0..3]; celld follows cellq in memory
  (void)celld;
  corrections_fused_kernel<<<RD_BLOCKS, RD_THREADS, 0, s>>>(cellq, K, hs, V, partial, ticket, corr);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_energy(const double* epart, int64_t count, double* partial, unsigned int* ticket, double* energy,
                          cudaStream_t s, int* nl) {
  energy_fused_kernel<<<RD_BLOCKS, RD_THREADS, 0, s>>>(epart, count, partial, ticket, energy);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_to_physical(bool fp64, const void* X, double* out, int p, int64_t K, double hs, int mode,
                               cudaStream_t s) {
  const int64_t n = (int64_t)(p + 1) * (p + 1) * K;
  const unsigned b = (unsigned)((n + 255) / 256);
  if (fp64)
    to_physical_kernel<double><<<b, 256, 0, s>>>((const double*)X, out, p, K, hs, mode);
  else
    to_physical_kernel<float><<<b, 256, 0, s>>>((const float*)X, out, p, K, hs, mode);
  return cudaGetLastError();
}

}  // namespace pmmm
