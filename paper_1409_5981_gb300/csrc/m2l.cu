// Per-wavevector M2L (Sec. 2.1: L~_k = G~_k M~_k) in the real-matrix form of
// App. A.8, one thread per (wavevector, output order l).  Spectra are stored
// channel-major ([c][k]), so the threads of a warp read consecutive k of a
// channel: every load and store is coalesced.  Several systems that share the
// kernel spectra are laid out [c][system][k] and taken by blockIdx.z.
#include "internal.cuh"
#include "translations.cuh"

namespace pmmm {

namespace {

// The output order l = blockIdx.y (uniform per block) selects a compile-time
// instance, so that only the terms m <= l of that order are issued.
template <int P, int L, typename T, class LM, class LG, class ST>
__device__ __forceinline__ void m2l_order_dispatch(int l, int p, LM&& Mk, LG&& Gk, ST&& St) {
  if (l == L) {
    m2l_order_l<P, L, T>(p, Mk, Gk, St);
    return;
  }
  if constexpr (L < P) m2l_order_dispatch<P, L + 1, T>(l, p, Mk, Gk, St);
}

// CT: the compile-time-order form (FP32, p <= 8).  Its eight order instances
// together exceed the instruction cache, so it pays only when each SM keeps to
// one order at a time, i.e. when one order alone fills the GPU (large meshes:
// the blocks of one order launch together); small meshes take the runtime form.
template <int P, typename T, bool CT>
__global__ void __launch_bounds__(128, (P <= 7 ? 4 : 1)) m2l_kernel(const cpx<T>* __restrict__ Mt, const cpx<T>* __restrict__ Gt,
                                                  cpx<T>* __restrict__ Lt, int64_t Kh, int nsys, int p) {
  const int l = blockIdx.y;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Kh) return;
  const int64_t cstride = (int64_t)nsys * Kh, mk0 = (int64_t)blockIdx.z * Kh + k;
  auto Mk = [&](int c) { return Mt[c * cstride + mk0]; };
  auto Gk = [&](int s) { return Gt[(int64_t)s * Kh + k]; };
  auto St = [&](int c, cpx<T> v) { Lt[c * cstride + mk0] = v; };
  if constexpr (CT)
    m2l_order_dispatch<P, 0, T>(l, p, Mk, Gk, St);
  else
    m2l_order<P, T>(l, p, Mk, Gk, St);
}

// Tile form: one block per tile of M2L_TILE consecutive wavevectors (of one
// system), holding the tile's spectra of all C moment channels and the
// parity-reduced kernel spectra (one real number per component, m2l_order_par) in
// shared memory (one coalesced asynchronous copy of each row), so that every
// spectrum value is read from memory once however many output orders use it.
// Warp w takes the output orders w and P - w for the 32 wavevectors of the tile
// (lane = wavevector): each warp then has the same number of terms, (P + 2)
// (lam + 1) per source order lam.  Stores are coalesced rows of the tile.
constexpr int M2L_TILE = 32;

template <int P, typename T>
constexpr int m2l_tile_threads() { return 32 * ((P + 2) / 2); }
template <int P, typename T>
constexpr size_t m2l_tile_smem() {
  return ((size_t)(P + 1) * (P + 1) * sizeof(cpx<T>) + (size_t)(2 * P + 1) * (2 * P + 1) * sizeof(T)) * M2L_TILE;
}

// 4-, 8- or 16-byte asynchronous copy global -> shared; zero fill when !valid
template <int BYTES>
__device__ __forceinline__ void cp_async_n(void* dst, const void* src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  const int n = valid ? BYTES : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src), "n"(BYTES), "r"(n) : "memory");
}

template <int P, typename T>
__global__ void __launch_bounds__(m2l_tile_threads<P, T>()) m2l_tile_kernel(const cpx<T>* __restrict__ Mt,
                                                                           const T* __restrict__ Gr,
                                                                           cpx<T>* __restrict__ Lt, int64_t Kh,
                                                                           int nsys) {
  constexpr int C = (P + 1) * (P + 1), CG = (2 * P + 1) * (2 * P + 1);
  extern __shared__ __align__(16) unsigned char m2l_smem[];
  cpx<T>* Ms = reinterpret_cast<cpx<T>*>(m2l_smem);
  T* Gs = reinterpret_cast<T*>(Ms + C * M2L_TILE);
  const int64_t k0 = (int64_t)blockIdx.x * M2L_TILE;
  const int64_t cstride = (int64_t)nsys * Kh, mk0 = (int64_t)blockIdx.y * Kh + k0;
  for (int i = threadIdx.x; i < (C + CG) * M2L_TILE; i += blockDim.x) {
    const int row = i / M2L_TILE, tk = i - row * M2L_TILE;
    const bool valid = k0 + tk < Kh;
    const int t = valid ? tk : 0;
    if (row < C)
      cp_async_n<sizeof(cpx<T>)>(Ms + i, Mt + row * cstride + mk0 + t, valid);
    else
      cp_async_n<sizeof(T)>(Gs + (i - C * M2L_TILE), Gr + (int64_t)(row - C) * Kh + k0 + t, valid);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const int tk = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool store = k0 + tk < Kh;
  cpx<T>* Lo = Lt + mk0 + tk;
  auto Mk = [&](int c) { return Ms[c * M2L_TILE + tk]; };
  auto Gk = [&](int s) { return Gs[s * M2L_TILE + tk]; };
  auto St = [&](int c, cpx<T> v) {
    if (store) Lo[c * cstride] = v;
  };
  m2l_order_par<P, T>(w, P, Mk, Gk, St);
  if (P - w != w) m2l_order_par<P, T>(P - w, P, Mk, Gk, St);
}

template <int P, typename T>
bool m2l_tile_fits() { return m2l_tile_smem<P, T>() <= 200 * 1024; }

template <int P, typename T>
cudaError_t run_tile(const void* Mt, const void* Gr, void* Lt, int64_t Kh, int nsys, cudaStream_t s) {
  const size_t smem = m2l_tile_smem<P, T>();
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(m2l_tile_kernel<P, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((unsigned)((Kh + M2L_TILE - 1) / M2L_TILE), (unsigned)nsys);
  m2l_tile_kernel<P, T><<<grid, m2l_tile_threads<P, T>(), smem, s>>>((const cpx<T>*)Mt, (const T*)Gr,
                                                                      (cpx<T>*)Lt, Kh, nsys);
  return cudaGetLastError();
}

// blocks of one order from which the compile-time form is taken (more than a wave of 4 x 152)
constexpr int64_t M2L_CT_MIN_BLOCKS = 1024;

template <int P, typename T>
cudaError_t run(const void* Mt, const void* Gt, const void* Gr, void* Lt, int64_t Kh, int nsys, cudaStream_t s) {
  if (Gr && m2l_tile_fits<P, T>()) return run_tile<P, T>(Mt, Gr, Lt, Kh, nsys, s);
  dim3 grid((unsigned)((Kh + 127) / 128), P + 1, (unsigned)nsys);
  const bool ct = sizeof(T) == 4 && P <= 8 && (int64_t)grid.x * nsys >= M2L_CT_MIN_BLOCKS;
  if constexpr (sizeof(T) == 4 && P <= 8) {
    if (ct) {
      m2l_kernel<P, T, true><<<grid, 128, 0, s>>>((const cpx<T>*)Mt, (const cpx<T>*)Gt, (cpx<T>*)Lt, Kh, nsys, P);
      return cudaGetLastError();
    }
  }
  m2l_kernel<P, T, false><<<grid, 128, 0, s>>>((const cpx<T>*)Mt, (const cpx<T>*)Gt, (cpx<T>*)Lt, Kh, nsys, P);
  return cudaGetLastError();
}

template <int P>
cudaError_t dispatch(int p, bool fp64, const void* Mt, const void* Gt, const void* Gr, void* Lt, int64_t Kh, int nsys,
                     cudaStream_t s) {
  if (p == P)
    return fp64 ? run<P, double>(Mt, Gt, Gr, Lt, Kh, nsys, s) : run<P, float>(Mt, Gt, Gr, Lt, Kh, nsys, s);
  if constexpr (P < PMMM_PMAX) return dispatch<P + 1>(p, fp64, Mt, Gt, Gr, Lt, Kh, nsys, s);
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_m2l(int p, bool fp64, const void* Mt, const void* Gt, const void* Gr, void* Lt, int64_t Kh,
                       cudaStream_t s, int* nl) {
  ++*nl;
  return dispatch<0>(p, fp64, Mt, Gt, Gr, Lt, Kh, 1, s);
}

cudaError_t launch_m2l_systems(int p, bool fp64, const void* Mt, const void* Gt, const void* Gr, void* Lt, int64_t Kh,
                               int nsys, cudaStream_t s, int* nl) {
  if (nsys < 1 || nsys > 65535) return cudaErrorInvalidValue;
  ++*nl;
  return dispatch<0>(p, fp64, Mt, Gt, Gr, Lt, Kh, nsys, s);
}

}  // namespace pmmm
