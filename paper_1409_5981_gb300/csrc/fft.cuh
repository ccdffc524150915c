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
