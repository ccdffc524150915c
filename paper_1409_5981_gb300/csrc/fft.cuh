// Radix-2/4/8 Stockham butterflies for power-of-two FFTs held in shared memory.
//
// Sign convention (the cell convolution of Sec. 2.1 and App. C): the forward
// transform is X_k = sum_j x_j exp(-2 pi i jk/L), the inverse uses exp(+2 pi i jk/L)
// without normalisation (the 1/K of the inverse is folded into the kernel spectra).
//
// A stage of radix R on a length-L transform, with Ns the product of the radices of
// the earlier stages, maps butterfly j (0 <= j < L/R) as
//   inputs  in[j + r L/R], r = 0..R-1, twiddled by w^(r (j mod Ns)), w = exp(-+2 pi i/(Ns R))
//   outputs out[(j - j mod Ns) R + (j mod Ns) + r Ns]
// which leaves the result in natural order after the last stage (autosort).
#pragma once
#include "common.cuh"

namespace pmmm {

struct FftPlan1D {
  int L;          // transform length (power of two, 2..512)
  int nst;        // number of stages
  int rad[10];    // radix of each stage (2, 4 or 8)
};

inline FftPlan1D make_fft_plan(int L) {
  FftPlan1D pl{};
  pl.L = L;
  int rem = L, n = 0;
  while (rem > 1) {
    int r = (rem % 8 == 0) ? 8 : (rem % 4 == 0 ? 4 : 2);
    pl.rad[n++] = r;
    rem /= r;
  }
  pl.nst = n;
  return pl;
}

// s = -1 forward, +1 inverse
template <typename T>
PMMM_HD void dft2(cpx<T>* v) {
  const cpx<T> a = v[0], b = v[1];
  v[0] = a + b;
  v[1] = a - b;
}

template <typename T>
PMMM_HD void dft4(cpx<T>* v, int s) {
  const cpx<T> a0 = v[0] + v[2], a1 = v[0] - v[2], a2 = v[1] + v[3], a3 = v[1] - v[3];
  const cpx<T> ia3 = mul_si(a3, s);  // (s i) a3
  v[0] = a0 + a2;
  v[2] = a0 - a2;
  v[1] = a1 + ia3;
  v[3] = a1 - ia3;
}

template <typename T>
PMMM_HD void dft8(cpx<T>* v, int s) {
  cpx<T> e[4] = {v[0], v[2], v[4], v[6]};
  cpx<T> o[4] = {v[1], v[3], v[5], v[7]};
  dft4(e, s);
  dft4(o, s);
  const T h = T(0.70710678118654752440084436210484903928483593768847);
  // w^k = exp(s i pi k/4): w^1 = h(1 + s i), w^2 = s i, w^3 = h(-1 + s i)
  const cpx<T> w1o = h * (o[1] + mul_si(o[1], s));
  const cpx<T> w2o = mul_si(o[2], s);
  const cpx<T> w3o = h * (mul_si(o[3], s) - o[3]);
  v[0] = e[0] + o[0];
  v[4] = e[0] - o[0];
  v[1] = e[1] + w1o;
  v[5] = e[1] - w1o;
  v[2] = e[2] + w2o;
  v[6] = e[2] - w2o;
  v[3] = e[3] + w3o;
  v[7] = e[3] - w3o;
}

// One butterfly of a Stockham stage; element t of a transform lives at in[t * es].
template <typename T, int R>
PMMM_HD void stockham_bf(const cpx<T>* in, cpx<T>* out, int L, int Ns, int j, int es, const cpx<T>* tw, int s) {
  const int k = j & (Ns - 1);
  cpx<T> v[R];
  const int q = L / R;
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = in[(j + r * q) * es];
  if (Ns > 1) {
    const int step = L / (Ns * R);
#pragma unroll
    for (int r = 1; r < R; ++r) {
      cpx<T> w = tw[r * k * step];  // exp(-2 pi i r k / (Ns R))
      if (s > 0) w = conjg(w);
      v[r] = v[r] * w;
    }
  }
  if (R == 2) dft2(v);
  if (R == 4) dft4(v, s);
  if (R == 8) dft8(v, s);
  const int base = (j - k) * R + k;
#pragma unroll
  for (int r = 0; r < R; ++r) out[(base + r * Ns) * es] = v[r];
}

template <typename T>
PMMM_HD void stockham_bf_any(int R, const cpx<T>* in, cpx<T>* out, int L, int Ns, int j, int es, const cpx<T>* tw,
                             int s) {
  if (R == 8) stockham_bf<T, 8>(in, out, L, Ns, j, es, tw, s);
  else if (R == 4) stockham_bf<T, 4>(in, out, L, Ns, j, es, tw, s);
  else stockham_bf<T, 2>(in, out, L, Ns, j, es, tw, s);
}

}  // namespace pmmm

#if defined(__CUDACC__)
namespace pmmm {

// ---------------------------------------------------------------------------
// The same Stockham stages with the length, the stage radices and the direction
// known at compile time (lengths 8 ... 512), so that every index and twiddle
// step folds into constants.  Radix of stage st of a length-L transform: 8 while
// the remaining length is a multiple of 8, then 4, then 2 (as make_fft_plan).
constexpr int ct_radix(int L, int st) {
  int rem = L, r = 2;
  for (int i = 0; i <= st; ++i) {
    r = (rem % 8 == 0) ? 8 : (rem % 4 == 0 ? 4 : 2);
    rem /= r;
  }
  return r;
}
constexpr int ct_nstages(int L) {
  int n = 0, rem = L;
  while (rem > 1) {
    rem /= (rem % 8 == 0) ? 8 : (rem % 4 == 0 ? 4 : 2);
    ++n;
  }
  return n;
}
constexpr int ct_ns(int L, int st) {
  int ns = 1;
  for (int i = 0; i < st; ++i) ns *= ct_radix(L, i);
  return ns;
}

// One butterfly of stage (R, NS) of a length-L transform, elements at in[t * es];
// tw[t] = exp(-2 pi i t / L) (the inverse, SGN = +1, uses the conjugates).
template <typename T, int L, int R, int NS, int SGN>
__device__ __forceinline__ void stockham_bf_ct(const cpx<T>* in, cpx<T>* out, int j, int es, const cpx<T>* tw) {
  constexpr int q = L / R;
  const int k = j & (NS - 1);
  cpx<T> v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = in[(j + r * q) * es];
  if constexpr (NS > 1) {
    constexpr int step = L / (NS * R);
#pragma unroll
    for (int r = 1; r < R; ++r) {
      cpx<T> w = tw[r * k * step];
      if constexpr (SGN > 0) w.y = -w.y;
      v[r] = v[r] * w;
    }
  }
  if constexpr (R == 2) dft2(v);
  if constexpr (R == 4) dft4(v, SGN);
  if constexpr (R == 8) dft8(v, SGN);
  const int base = (j - k) * R + k;
#pragma unroll
  for (int r = 0; r < R; ++r) out[(base + r * NS) * es] = v[r];
}

// Every stage of `ntrans` length-L transforms held in shared memory (A -> B ->
// ..., the result ends in A on return, pointers swapped as in run_stages).
// ROWS: transform tr at A[tr L ...] (stride 1); else element t of transform tr at
// A[t es + tr], es = ntrans unless given (a larger, odd stride keeps the lanes of
// a warp on distinct banks when ntrans is a power of two).  Block-wide: ends
// with __syncthreads().
template <typename T, bool ROWS, int L, int SGN, int ST = 0>
__device__ __forceinline__ void run_stages_ct(cpx<T>*& A, cpx<T>*& B, int ntrans, const cpx<T>* tw, int es = 0) {
  if (es == 0) es = ntrans;
  if constexpr (ST < ct_nstages(L)) {
    constexpr int R = ct_radix(L, ST), NS = ct_ns(L, ST), nb = L / R;
    if constexpr (ROWS) {
      for (int t = threadIdx.x; t < nb * ntrans; t += blockDim.x) {
        const int tr = t / nb, j = t % nb;
        stockham_bf_ct<T, L, R, NS, SGN>(A + tr * L, B + tr * L, j, 1, tw);
      }
    } else {
      // t = j ntrans + tr, walked with an incremental (tr, j) to avoid a division per task
      const int dq = (int)blockDim.x / ntrans, dr = (int)blockDim.x - dq * ntrans;
      int tr = (int)threadIdx.x % ntrans, j = (int)threadIdx.x / ntrans;
      for (; j < nb; j += dq) {
        stockham_bf_ct<T, L, R, NS, SGN>(A + tr, B + tr, j, es, tw);
        tr += dr;
        if (tr >= ntrans) {
          tr -= ntrans;
          ++j;
        }
      }
    }
    __syncthreads();
    cpx<T>* tmp = A;
    A = B;
    B = tmp;
    run_stages_ct<T, ROWS, L, SGN, ST + 1>(A, B, ntrans, tw, es);
  }
}

}  // namespace pmmm
#endif  // __CUDACC__
