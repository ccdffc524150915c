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

// ---------------------------------------------------------------------------
// FP32 packed form of m2l_order_par: the real and imaginary parts of every
// spectrum value travel together as a float2, each kernel scalar g is used as the
// pair (g, g), and the sums and multiply-adds run as packed f32x2 operations, so a
// term (m, mu > 0) issues 4 packed additions and 4 packed multiply-adds instead of
// 4 additions and 8 multiply-adds.  Same operations per component, same order.
__device__ __forceinline__ float2 pk_neg(float2 a) { return make_float2(-a.x, -a.y); }
// SA X + SB Y for compile-time signs
template <int SA, int SB>
__device__ __forceinline__ float2 pk_comb(float2 X, float2 Y) {
  if constexpr (SA > 0 && SB > 0) return __fadd2_rn(X, Y);
  if constexpr (SA > 0 && SB < 0) return __fadd2_rn(X, pk_neg(Y));
  if constexpr (SA < 0 && SB > 0) return __fadd2_rn(Y, pk_neg(X));
  return pk_neg(__fadd2_rn(X, Y));
}
// spectrum scalar of Re S_j^KAP (SRe) or Im S_j^KAP (SIm) as (index into the stored
// components, sign), from sre[a] = X[sidx(j, a)], sim[a] = X[sidx(j, -a)], a >= 0
template <int KAP> struct SRe { static constexpr int idx = KAP >= 0 ? KAP : -KAP, sgn = (KAP < 0 && ((-KAP) & 1)) ? -1 : 1; };
template <int KAP> struct SIm { static constexpr int idx = KAP >= 0 ? KAP : -KAP, sgn = (KAP < 0 && !((-KAP) & 1)) ? -1 : 1, zero = KAP == 0; };
template <int P, int M, int MU>
__device__ __forceinline__ void m2l_term_pk(const float2* sre, const float2* sim, const float2* mre, const float2* mim,
                                            float2* Lre, float2* Lim) {
  using A = SRe<-(M + MU)>;
  using B = SIm<-(M + MU)>;
  if constexpr (MU == 0) {
    Lre[M] = __ffma2_rn(A::sgn > 0 ? sre[A::idx] : pk_neg(sre[A::idx]), mre[0], Lre[M]);
    if constexpr (!B::zero) Lim[M] = __ffma2_rn(B::sgn > 0 ? sim[B::idx] : pk_neg(sim[B::idx]), mre[0], Lim[M]);
  } else {
    using Cc = SRe<MU - M>;
    using Dd = SIm<MU - M>;
    constexpr int cs = (MU & 1) ? -Cc::sgn : Cc::sgn, ds = (MU & 1) ? -Dd::sgn : Dd::sgn;
    const float2 a = sre[A::idx], c = sre[Cc::idx];
    const float2 u1 = pk_comb<A::sgn, cs>(a, c);
    const float2 u4 = pk_comb<A::sgn, -cs>(a, c);
    float2 u2, u3;
    if constexpr (B::zero && Dd::zero) {
      u2 = make_float2(0.f, 0.f);
      u3 = u2;
    } else if constexpr (B::zero) {
      u2 = ds > 0 ? sim[Dd::idx] : pk_neg(sim[Dd::idx]);
      u3 = u2;
    } else if constexpr (Dd::zero) {
      u2 = B::sgn > 0 ? pk_neg(sim[B::idx]) : sim[B::idx];
      u3 = B::sgn > 0 ? sim[B::idx] : pk_neg(sim[B::idx]);
    } else {
      u2 = pk_comb<ds, -B::sgn>(sim[Dd::idx], sim[B::idx]);
      u3 = pk_comb<B::sgn, ds>(sim[B::idx], sim[Dd::idx]);
    }
    Lre[M] = __ffma2_rn(u1, mre[MU], Lre[M]);
    if constexpr (!(B::zero && Dd::zero)) Lre[M] = __ffma2_rn(u2, mim[MU], Lre[M]);
    if constexpr (!(B::zero && Dd::zero)) Lim[M] = __ffma2_rn(u3, mre[MU], Lim[M]);
    Lim[M] = __ffma2_rn(u4, mim[MU], Lim[M]);
  }
}
template <int P, int M, int MU>
struct M2LColPk {
  __device__ __forceinline__ static void apply(int l, const float2* sre, const float2* sim, const float2* mre,
                                               const float2* mim, float2* Lre, float2* Lim) {
    if (M > l) return;
    m2l_term_pk<P, M, MU>(sre, sim, mre, mim, Lre, Lim);
    if constexpr (M < P) M2LColPk<P, M + 1, MU>::apply(l, sre, sim, mre, mim, Lre, Lim);
  }
};
template <int P, int MU>
struct M2LColsPk {
  __device__ __forceinline__ static void apply(int l, int lam, const float2* sre, const float2* sim,
                                               const float2* mre, const float2* mim, float2* Lre, float2* Lim) {
    if (MU > lam) return;
    M2LColPk<P, 0, MU>::apply(l, sre, sim, mre, mim, Lre, Lim);
    if constexpr (MU < P) M2LColsPk<P, MU + 1>::apply(l, lam, sre, sim, mre, mim, Lre, Lim);
  }
};
// One output order l at one wavevector: Mk(c) -> float2 spectrum of channel c,
// Gs1(s) -> the parity-reduced kernel scalar of component s, St(c, float2).
template <int P, class LM, class LG, class ST>
__device__ __forceinline__ void m2l_order_pk(int l, int p, LM&& Mk, LG&& Gs1, ST&& St) {
  float2 Lre[P + 1], Lim[P + 1];
#pragma unroll
  for (int m = 0; m <= P; ++m) Lre[m] = Lim[m] = make_float2(0.f, 0.f);
  for (int lam = 0; lam <= p; ++lam) {
    const int j = l + lam;
    const bool odd = (j & 1) != 0;
    float2 mre[P + 1], mim[P + 1];
#pragma unroll
    for (int mu = 0; mu <= P; ++mu) {
      if (mu <= lam) {
        float2 v = Mk(sidx(lam, mu));
        mre[mu] = odd ? make_float2(-v.y, v.x) : v;
        if (mu > 0) {
          v = Mk(sidx(lam, -mu));
          mim[mu] = odd ? make_float2(-v.y, v.x) : v;
        }
      }
    }
    float2 sre[2 * P + 1], sim[2 * P + 1];
#pragma unroll
    for (int a = 0; a <= 2 * P; ++a) {
      if (a <= j) {
        const float g = Gs1(sidx(j, a));
        sre[a] = make_float2(g, g);
        if (a > 0) {
          const float h = Gs1(sidx(j, -a));
          sim[a] = make_float2(h, h);
        }
      }
    }
    M2LColsPk<P, 0>::apply(l, lam, sre, sim, mre, mim, Lre, Lim);
  }
#pragma unroll
  for (int m = 0; m <= P; ++m) {
    if (m <= l) {
      St(sidx(l, m), Lre[m]);
      if (m > 0) St(sidx(l, -m), Lim[m]);
    }
  }
}

// Tile form: one block per tile of M2L_TILE consecutive wavevectors (of one
// system), holding the tile's spectra of all C moment channels and the
// parity-reduced kernel spectra (one real number per component; m2l_order_pk in
// FP32, m2l_order_par in FP64) in shared memory (one coalesced asynchronous copy of each row), so that every
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
__global__ void __launch_bounds__(m2l_tile_threads<P, T>(), (sizeof(T) == 4 ? 4 : 1)) m2l_tile_kernel(const cpx<T>* __restrict__ Mt,
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
  if constexpr (sizeof(T) == 4) {
    const float2* M2 = reinterpret_cast<const float2*>(Ms);
    auto Mk = [&](int c) { return M2[c * M2L_TILE + tk]; };
    auto Gk = [&](int s) { return (float)Gs[s * M2L_TILE + tk]; };
    auto St = [&](int c, float2 v) {
      if (store) Lo[c * cstride] = mk((T)v.x, (T)v.y);
    };
    m2l_order_pk<P>(w, P, Mk, Gk, St);
    if (P - w != w) m2l_order_pk<P>(P - w, P, Mk, Gk, St);
  } else {
    auto Mk = [&](int c) { return Ms[c * M2L_TILE + tk]; };
    auto Gk = [&](int s) { return Gs[s * M2L_TILE + tk]; };
    auto St = [&](int c, cpx<T> v) {
      if (store) Lo[c * cstride] = v;
    };
    m2l_order_par<P, T>(w, P, Mk, Gk, St);
    if (P - w != w) m2l_order_par<P, T>(P - w, P, Mk, Gk, St);
  }
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
