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

// blocks of one order from which the compile-time form is taken (more than a wave of 4 x 152)
constexpr int64_t M2L_CT_MIN_BLOCKS = 1024;

template <int P, typename T>
cudaError_t run(const void* Mt, const void* Gt, void* Lt, int64_t Kh, int nsys, cudaStream_t s) {
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
cudaError_t dispatch(int p, bool fp64, const void* Mt, const void* Gt, void* Lt, int64_t Kh, int nsys,
                     cudaStream_t s) {
  if (p == P) return fp64 ? run<P, double>(Mt, Gt, Lt, Kh, nsys, s) : run<P, float>(Mt, Gt, Lt, Kh, nsys, s);
  if constexpr (P < PMMM_PMAX) return dispatch<P + 1>(p, fp64, Mt, Gt, Lt, Kh, nsys, s);
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_m2l(int p, bool fp64, const void* Mt, const void* Gt, void* Lt, int64_t Kh, cudaStream_t s,
                       int* nl) {
  ++*nl;
  return dispatch<0>(p, fp64, Mt, Gt, Lt, Kh, 1, s);
}

cudaError_t launch_m2l_systems(int p, bool fp64, const void* Mt, const void* Gt, void* Lt, int64_t Kh, int nsys,
                               cudaStream_t s, int* nl) {
  if (nsys < 1 || nsys > 65535) return cudaErrorInvalidValue;
  ++*nl;
  return dispatch<0>(p, fp64, Mt, Gt, Lt, Kh, nsys, s);
}

}  // namespace pmmm
