// Batched form: many independent systems that share one plan (box, mesh, p,
// boundary).  The systems are laid side by side as one mesh of B*K cells
// (system s owns cells s*K ... s*K + K - 1), so binning, sorting, P2M, the FFTs
// (C*B channels), L2P and the near field run once over all systems.  Per
// wavevector the M2L of all systems is one complex matrix product
//   L~(k)[C x B] = A~(k)[C x C] M~(k)[C x B]
// (Sec. 2.1 convolution theorem with the real-matrix form of App. A.8), with
// A~(k) assembled once per k from the (2p+1)^2 kernel spectra.
#include <algorithm>
#include <vector>

#include "binning.cuh"
#include "internal.cuh"
#include "m2l_table.cuh"

namespace pmmm {

namespace {

constexpr double kPi = 3.14159265358979323846;

// system of particle i: offsets[s] <= i < offsets[s+1]
__device__ __forceinline__ int system_of(const int64_t* __restrict__ off, int nsys, int64_t i) {
  int lo = 0, hi = nsys;  // invariant: off[lo] <= i < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <typename T>
__global__ void bin_batched_kernel(const T* __restrict__ pos, const T* __restrict__ q, int64_t n,
                                   const int64_t* __restrict__ offsets, int nsys, Geo g, int64_t Ksys,
                                   uint32_t* __restrict__ keys, T* __restrict__ rec, int* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = system_of(offsets, nsys, i);
  bin_record<T>(pos, q, i, g, (uint32_t)((int64_t)s * Ksys), keys, rec, err);
}

// Batched M2L on wavevector-major spectra ([k][c][system]): block = KT
// consecutive wavevectors x BT systems.  Shared memory:
// Ms[c][kt][b] (M~ in, L~ out), At[c_in][c_out] (A~ of the current k), g[s].
// Thread tiles of 4 output channels x 4 systems.
template <typename T, int KT>
__global__ void __launch_bounds__(256) m2l_batched_kernel(const cpx<T>* __restrict__ Mt, const cpx<T>* __restrict__ Gt,
                                                          cpx<T>* __restrict__ Lt, const int4* __restrict__ tab, int C,
                                                          int CG, int B, int BT, int64_t Kh) {
  extern __shared__ unsigned char smem_raw[];
  cpx<T>* Ms = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* At = Ms + (size_t)C * KT * BT;
  cpx<T>* gk = At + (size_t)C * C;
  const int64_t k0 = (int64_t)blockIdx.x * KT;
  const int kc = (int)min((int64_t)KT, Kh - k0);
  const int b0 = blockIdx.y * BT;
  const int nb = min(BT, B - b0);
  const int tid = threadIdx.x;
  // M~ tile: element (c, b, kt) of system b0 + b at Mt[((k0 + kt)*C + c)*B + b0 + b]
  // (wavevector-major spectra: consecutive threads read consecutive systems)
  for (int idx = tid; idx < C * nb * KT; idx += blockDim.x) {
    const int b = idx % nb, ck = idx / nb, c = ck % C, kt = ck / C;
    cpx<T> v = mk(T(0), T(0));
    if (kt < kc) v = Mt[((k0 + kt) * C + c) * B + b0 + b];
    Ms[((size_t)c * KT + kt) * BT + b] = v;
  }
  const int ntc = (C + 3) / 4, ntb = (nb + 3) / 4, ntile = ntc * ntb;
  for (int kt = 0; kt < kc; ++kt) {
    for (int s = tid; s < CG; s += blockDim.x) gk[s] = Gt[(int64_t)s * Kh + k0 + kt];
    __syncthreads();
    for (int e = tid; e < C * C; e += blockDim.x) {
      const int4 t = tab[e];  // e = c_out * C + c_in
      const cpx<T> a = mk((T)t.y * gk[t.x].x + (T)t.w * gk[t.z].x, (T)t.y * gk[t.x].y + (T)t.w * gk[t.z].y);
      const int co = e / C, ci = e - co * C;
      At[(size_t)ci * C + co] = a;
    }
    __syncthreads();
    cpx<T> acc[4][4];
    int ct = 0, bt = 0;
    const bool has = tid < ntile;  // one tile per thread (ntile <= blockDim for C <= 64, BT <= 64)
    if (has) {
      ct = tid % ntc;
      bt = tid / ntc;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = mk(T(0), T(0));
      for (int ci = 0; ci < C; ++ci) {
        cpx<T> a[4], m[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int co = 4 * ct + i;
          a[i] = co < C ? At[(size_t)ci * C + co] : mk(T(0), T(0));
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int b = 4 * bt + j;
          m[j] = b < nb ? Ms[((size_t)ci * KT + kt) * BT + b] : mk(T(0), T(0));
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) cmac(acc[i][j], a[i], m[j]);
      }
    }
    __syncthreads();  // every thread has read M~(kt) and A~
    if (has) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int co = 4 * ct + i, b = 4 * bt + j;
          if (co < C && b < nb) Ms[((size_t)co * KT + kt) * BT + b] = acc[i][j];
        }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < C * nb * KT; idx += blockDim.x) {
    const int b = idx % nb, ck = idx / nb, c = ck % C, kt = ck / C;
    if (kt < kc) Lt[((k0 + kt) * C + c) * B + b0 + b] = Ms[((size_t)c * KT + kt) * BT + b];
  }
}

// Per-system periodic corrections (App. B.3) in two fixed-order levels: block
// (chunk, s) sums the five per-cell FP64 quantities of RB_CHUNK cells of system
// s; one block per system then sums its chunks and writes corr[16 s + ...] as in
// the single-system kernel.
constexpr int RB_CHUNK = 4096;

template <int NQ>
__device__ __forceinline__ void block_sum(double (&acc)[NQ], double (*sh)[256]) {
#pragma unroll
  for (int qn = 0; qn < NQ; ++qn) sh[qn][threadIdx.x] = acc[qn];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int qn = 0; qn < NQ; ++qn) sh[qn][threadIdx.x] += sh[qn][threadIdx.x + w];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) cellsum_partial_kernel(const double* __restrict__ cellsum, int64_t Ktot,
                                                              int64_t Ksys, int nchunk, double* __restrict__ part) {
  __shared__ double sh[5][256];
  const int s = blockIdx.y, ch = blockIdx.x;
  const int64_t lo = (int64_t)s * Ksys + (int64_t)ch * RB_CHUNK;
  const int64_t hi = min(lo + RB_CHUNK, (int64_t)(s + 1) * Ksys);
  double acc[5] = {0, 0, 0, 0, 0};
  for (int64_t c = lo + threadIdx.x; c < hi; c += blockDim.x)
#pragma unroll
    for (int qn = 0; qn < 5; ++qn) acc[qn] += cellsum[qn * Ktot + c];
  block_sum<5>(acc, sh);
  if (threadIdx.x < 5) part[((int64_t)s * nchunk + ch) * 5 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(256) corrections_batched_kernel(const double* __restrict__ part, int nchunk,
                                                                  double hs, double V, double* __restrict__ corr) {
  __shared__ double sh[5][256];
  const int s = blockIdx.x;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int ch = threadIdx.x; ch < nchunk; ch += blockDim.x)
#pragma unroll
    for (int qn = 0; qn < 5; ++qn) acc[qn] += part[((int64_t)s * nchunk + ch) * 5 + qn];
  block_sum<5>(acc, sh);
  if (threadIdx.x == 0) {
    const double f = 2.0 * kPi / (3.0 * V);
    double* c = corr + 16 * s;
    c[0] = f * sh[4][0] * hs * hs;
    c[1] = -2.0 * f * sh[1][0] * hs;
    c[2] = -2.0 * f * sh[2][0] * hs;
    c[3] = -2.0 * f * sh[3][0] * hs;
    c[4] = f * sh[0][0];
    corr_store_f32(c);
    for (int qn = 0; qn < 5; ++qn) c[8 + qn] = sh[qn][0];
  }
}

// Per-system energy and net force from the near-field work items (numbered in
// cell order): block (chunk, s) sums RB_CHUNK items of system s, then one block
// per system sums its chunks.  The item range of system s is
// item_start[s Ksys] ... item_start[(s+1) Ksys].
__global__ void __launch_bounds__(256) energy_partial_kernel(const double* __restrict__ epart,
                                                             const uint32_t* __restrict__ item_start, int64_t Ksys,
                                                             int nchunk, double* __restrict__ part) {
  __shared__ double sh[4][256];
  const int s = blockIdx.y, ch = blockIdx.x;
  const int64_t b = item_start[(int64_t)s * Ksys], e = item_start[(int64_t)(s + 1) * Ksys];
  double acc[4] = {0, 0, 0, 0};
  const int64_t lo = b + (int64_t)ch * RB_CHUNK, hi = min(lo + RB_CHUNK, e);
  for (int64_t it = lo + threadIdx.x; it < hi; it += blockDim.x)
#pragma unroll
    for (int qn = 0; qn < 4; ++qn) acc[qn] += epart[4 * it + qn];
  block_sum<4>(acc, sh);
  if (threadIdx.x < 4) part[((int64_t)s * nchunk + ch) * 4 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(256) energy_batched_kernel(const double* __restrict__ part, int nchunk,
                                                             double* __restrict__ energies) {
  __shared__ double sh[4][256];
  const int s = blockIdx.x;
  double acc[4] = {0, 0, 0, 0};
  for (int ch = threadIdx.x; ch < nchunk; ch += blockDim.x)
#pragma unroll
    for (int qn = 0; qn < 4; ++qn) acc[qn] += part[((int64_t)s * nchunk + ch) * 4 + qn];
  block_sum<4>(acc, sh);
  if (threadIdx.x < 4) energies[4 * s + threadIdx.x] = sh[threadIdx.x][0];
}

template <typename T>
__global__ void __launch_bounds__(256) transpose_kernel(const cpx<T>* __restrict__ in, cpx<T>* __restrict__ out,
                                                        int64_t R, int64_t Kh) {
  __shared__ cpx<T> tile[32][33];
  const int64_t nk = (Kh + 31) / 32;  // tiles along k (fastest), then along r
  const int64_t k0 = ((int64_t)blockIdx.x % nk) * 32, r0 = ((int64_t)blockIdx.x / nk) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int j = ty; j < 32; j += 8) {
    const int64_t r = r0 + j, k = k0 + tx;
    if (r < R && k < Kh) tile[j][tx] = in[r * Kh + k];
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int64_t k = k0 + j, r = r0 + tx;
    if (r < R && k < Kh) out[k * R + r] = tile[tx][j];
  }
}

template <typename T>
size_t m2l_batched_smem(int C, int CG, int KT, int BT) {
  return sizeof(cpx<T>) * ((size_t)C * KT * BT + (size_t)C * C + (size_t)CG);
}

template <typename T, int KT>
cudaError_t m2l_batched_run(const void* Mt, const void* Gt, void* Lt, const int4* tab, int C, int CG, int B, int BT,
                            int64_t Kh, cudaStream_t s) {
  const size_t smem = m2l_batched_smem<T>(C, CG, KT, BT);
  cudaError_t e = cudaFuncSetAttribute(m2l_batched_kernel<T, KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((Kh + KT - 1) / KT), (unsigned)((B + BT - 1) / BT));
  m2l_batched_kernel<T, KT><<<grid, 256, smem, s>>>((const cpx<T>*)Mt, (const cpx<T>*)Gt, (cpx<T>*)Lt, tab, C, CG, B,
                                                    BT, Kh);
  return cudaGetLastError();
}

}  // namespace

std::vector<int> build_m2l_table_int4(int p) {
  std::vector<M2LEntry> t = build_m2l_table(p);
  std::vector<int> out(4 * t.size());
  for (size_t i = 0; i < t.size(); ++i) {
    out[4 * i] = t[i].i1;
    out[4 * i + 1] = t[i].s1;
    out[4 * i + 2] = t[i].i2;
    out[4 * i + 3] = t[i].s2;
  }
  return out;
}

cudaError_t launch_bin_batched(const void* pos, const void* q, bool fp64, int64_t n, const int64_t* offsets, int nsys,
                               const Geo& g, int64_t Ksys, uint32_t* keys, void* rec, int* err, cudaStream_t s,
                               int* nl) {
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (fp64)
    bin_batched_kernel<double><<<blocks, 256, 0, s>>>((const double*)pos, (const double*)q, n, offsets, nsys, g, Ksys,
                                                      keys, (double*)rec, err);
  else
    bin_batched_kernel<float><<<blocks, 256, 0, s>>>((const float*)pos, (const float*)q, n, offsets, nsys, g, Ksys,
                                                     keys, (float*)rec, err);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_transpose(bool fp64, const void* in, void* out, int64_t R, int64_t Kh, cudaStream_t s, int* nl) {
  if (R <= 0 || Kh <= 0) return cudaSuccess;
  const int64_t tiles = ((Kh + 31) / 32) * ((R + 31) / 32);
  if (tiles > 0x7fffffff) return cudaErrorInvalidConfiguration;
  const unsigned grid = (unsigned)tiles;
  if (fp64)
    transpose_kernel<double><<<grid, 256, 0, s>>>((const cpx<double>*)in, (cpx<double>*)out, R, Kh);
  else
    transpose_kernel<float><<<grid, 256, 0, s>>>((const cpx<float>*)in, (cpx<float>*)out, R, Kh);
  ++*nl;
  return cudaGetLastError();
}

namespace {
// systems per block of the SIMT matrix product, or 0 when A~ does not fit
int m2l_batched_bt(bool fp64, int p, int B) {
  const int C = (p + 1) * (p + 1), CG = (2 * p + 1) * (2 * p + 1);
  const size_t cap = 200 * 1024;
  const size_t esz = fp64 ? sizeof(cpx<double>) : sizeof(cpx<float>);
  int BT = B;
  while (BT > 4 && ((C + 3) / 4) * ((BT + 3) / 4) > 256) BT = (BT + 1) / 2;
  while (BT > 1 && esz * ((size_t)C * BT + (size_t)C * C + CG) > cap) BT = (BT + 1) / 2;
  if (esz * ((size_t)C * BT + (size_t)C * C + CG) > cap || BT < 4) return 0;
  return BT;
}
}  // namespace

bool m2l_batched_gemm(bool fp64, int p, int B) { return m2l_batched_bt(fp64, p, B) > 0; }

// Chooses the wavevectors per block (KT) and systems per block (BT) that fit
// the shared memory and the one-tile-per-thread layout (C/4 * BT/4 <= 256).
// Spectra are wavevector-major; m2l_batched_gemm() tells whether it applies.
cudaError_t launch_m2l_batched(bool fp64, const void* Mt, const void* Gt, void* Lt, const int* tab, int p, int B,
                               int64_t Kh, cudaStream_t s, int* nl) {
  const int C = (p + 1) * (p + 1), CG = (2 * p + 1) * (2 * p + 1);
  const size_t cap = 200 * 1024;
  const int BT = m2l_batched_bt(fp64, p, B);
  if (BT == 0) return cudaErrorInvalidConfiguration;
  const size_t esz = fp64 ? sizeof(cpx<double>) : sizeof(cpx<float>);
  auto fits = [&](int KT, int bt) { return esz * ((size_t)C * KT * bt + (size_t)C * C + CG) <= cap; };
  ++*nl;
  const int4* t4 = (const int4*)tab;
  if (fits(4, BT))
    return fp64 ? m2l_batched_run<double, 4>(Mt, Gt, Lt, t4, C, CG, B, BT, Kh, s)
                : m2l_batched_run<float, 4>(Mt, Gt, Lt, t4, C, CG, B, BT, Kh, s);
  if (fits(2, BT))
    return fp64 ? m2l_batched_run<double, 2>(Mt, Gt, Lt, t4, C, CG, B, BT, Kh, s)
                : m2l_batched_run<float, 2>(Mt, Gt, Lt, t4, C, CG, B, BT, Kh, s);
  return fp64 ? m2l_batched_run<double, 1>(Mt, Gt, Lt, t4, C, CG, B, BT, Kh, s)
              : m2l_batched_run<float, 1>(Mt, Gt, Lt, t4, C, CG, B, BT, Kh, s);
}

int reduce_batched_chunks(int64_t Ksys, int64_t max_items_per_sys) {
  const int64_t m = std::max<int64_t>(Ksys, max_items_per_sys);
  return (int)std::max<int64_t>(1, (m + RB_CHUNK - 1) / RB_CHUNK);
}

cudaError_t launch_corrections_batched(const double* cellsum, int64_t Ktot, int64_t Ksys, int nsys, double hs, double V,
                                       double* partial, double* corr, cudaStream_t s, int* nl) {
  const int nchunk = (int)((Ksys + RB_CHUNK - 1) / RB_CHUNK);
  cellsum_partial_kernel<<<dim3((unsigned)nchunk, (unsigned)nsys), 256, 0, s>>>(cellsum, Ktot, Ksys, nchunk, partial);
  corrections_batched_kernel<<<nsys, 256, 0, s>>>(partial, nchunk, hs, V, corr);
  *nl += 2;
  return cudaGetLastError();
}

cudaError_t launch_energy_batched(const double* epart, const uint32_t* item_start, int64_t Ksys, int nsys, int nchunk,
                                  double* partial, double* energies, cudaStream_t s, int* nl) {
  energy_partial_kernel<<<dim3((unsigned)nchunk, (unsigned)nsys), 256, 0, s>>>(epart, item_start, Ksys, nchunk,
                                                                               partial);
  energy_batched_kernel<<<nsys, 256, 0, s>>>(partial, nchunk, energies);
  *nl += 2;
  return cudaGetLastError();
}

}  // namespace pmmm
