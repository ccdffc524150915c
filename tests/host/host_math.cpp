// Host build of the GPU library's per-element math headers, for CPU unit tests.
// Compiled by tests/test_host_math.py with g++; exposes plain C entry points.
#include <vector>
#include <cmath>
#include "common.cuh"
#include "harmonics.cuh"
#include "translations.cuh"
#include "fft.cuh"
#include "m2l_table.cuh"

using namespace pmmm;

template <int P>
static void reg_dispatch(int p, double x, double y, double z, double* out) {
  if (p == P) {
    regular_real<P, double>(x, y, z, out);
    return;
  }
  if constexpr (P < PMMM_PMAX) reg_dispatch<P + 1>(p, x, y, z, out);
}

template <int P>
static void m2l_dispatch(int p, const double* M, const double* G, double* L) {
  if (p == P) {
    const cpx<double>* Mc = reinterpret_cast<const cpx<double>*>(M);
    const cpx<double>* Gc = reinterpret_cast<const cpx<double>*>(G);
    cpx<double>* Lc = reinterpret_cast<cpx<double>*>(L);
    for (int l = 0; l <= p; ++l)
      m2l_order<P, double>(l, p, [&](int c) { return Mc[c]; }, [&](int s) { return Gc[s]; },
                           [&](int c, cpx<double> v) { Lc[c] = v; });
    return;
  }
  if constexpr (P < PMMM_PMAX) m2l_dispatch<P + 1>(p, M, G, L);
}

template <int P>
static void m2l_par_dispatch(int p, const double* M, const double* Gr, double* L) {
  if (p == P) {
    const cpx<double>* Mc = reinterpret_cast<const cpx<double>*>(M);
    cpx<double>* Lc = reinterpret_cast<cpx<double>*>(L);
    for (int l = 0; l <= p; ++l)
      m2l_order_par<P, double>(l, p, [&](int c) { return Mc[c]; }, [&](int s) { return Gr[s]; },
                               [&](int c, cpx<double> v) { Lc[c] = v; });
    return;
  }
  if constexpr (P < PMMM_PMAX) m2l_par_dispatch<P + 1>(p, M, Gr, L);
}

template <int P>
static void l2p_dispatch(int p, const double* L, const double* u, double* out) {
  if (p == P) {
    double R[(P + 1) * (P + 1)];
    regular_real<P, double>(u[0], u[1], u[2], R);
    double f, gx, gy, gz;
    l2p_real<P, double>([&](int c) { return L[c]; }, R, f, gx, gy, gz);
    out[0] = f; out[1] = gx; out[2] = gy; out[3] = gz;
    return;
  }
  if constexpr (P < PMMM_PMAX) l2p_dispatch<P + 1>(p, L, u, out);
}

template <int P>
static void l2p_stream_dispatch(int p, const double* L, const double* u, double* out) {
  if (p == P) {
    double f, gx, gy, gz;
    l2p_stream<P, double>([&](int c) { return L[c]; }, u[0], u[1], u[2], f, gx, gy, gz);
    out[0] = f; out[1] = gx; out[2] = gy; out[3] = gz;
    return;
  }
  if constexpr (P < PMMM_PMAX) l2p_stream_dispatch<P + 1>(p, L, u, out);
}

template <int P>
static void reg_stream_dispatch(int p, double x, double y, double z, double* out) {
  if (p == P) {
    regular_stream<P, double>(x, y, z, [&](int l, int m, double re, double im) {
      out[sidx(l, m)] = re;
      if (m > 0) out[sidx(l, -m)] = im;
    });
    return;
  }
  if constexpr (P < PMMM_PMAX) reg_stream_dispatch<P + 1>(p, x, y, z, out);
}

template <typename T>
static void fft_run(int L, int inverse, double* data) {
  FftPlan1D pl = make_fft_plan(L);
  std::vector<cpx<T>> a(L), b(L), tw(L);
  for (int t = 0; t < L; ++t) {
    double ang = -2.0 * M_PI * t / L;
    tw[t] = mk<T>((T)cos(ang), (T)sin(ang));
    a[t] = mk<T>((T)data[2 * t], (T)data[2 * t + 1]);
  }
  int Ns = 1;
  const int s = inverse ? 1 : -1;
  for (int st = 0; st < pl.nst; ++st) {
    int R = pl.rad[st];
    for (int j = 0; j < L / R; ++j) stockham_bf_any<T>(R, a.data(), b.data(), L, Ns, j, 1, tw.data(), s);
    std::swap(a, b);
    Ns *= R;
  }
  for (int t = 0; t < L; ++t) {
    data[2 * t] = a[t].x;
    data[2 * t + 1] = a[t].y;
  }
}

extern "C" {
// M2L of one wavevector from the parity-reduced kernel spectra (one real number per component)
void h_m2l_k_par(int p, const double* M, const double* Gr, double* L) { m2l_par_dispatch<0>(p, M, Gr, L); }
int h_pmax() { return PMMM_PMAX; }
void h_regular_real(int p, double x, double y, double z, double* out) { reg_dispatch<0>(p, x, y, z, out); }
void h_singular_real(int J, double x, double y, double z, double* out) {
  for (int m = 0; m <= J; ++m)
    singular_column<double>(m, J, x, y, z, [&](int l, double re, double im) {
      out[sidx(l, m)] = re;
      if (m > 0) out[sidx(l, -m)] = im;
    });
}
void h_fft(int L, int inverse, int single, double* data) {
  if (single) fft_run<float>(L, inverse, data);
  else fft_run<double>(L, inverse, data);
}
void h_m2l_k(int p, const double* M, const double* G, double* L) { m2l_dispatch<0>(p, M, G, L); }
void h_l2p(int p, const double* L, const double* u, double* out) { l2p_dispatch<0>(p, L, u, out); }
void h_l2p_stream(int p, const double* L, const double* u, double* out) { l2p_stream_dispatch<0>(p, L, u, out); }
void h_regular_stream(int p, double x, double y, double z, double* out) { reg_stream_dispatch<0>(p, x, y, z, out); }
// L = A M with A built from the entry table (complex k-space values)
void h_m2l_table(int p, const double* M, const double* G, double* L) {
  const int C = (p + 1) * (p + 1);
  std::vector<M2LEntry> t = build_m2l_table(p);
  for (int co = 0; co < C; ++co) {
    double re = 0, im = 0;
    for (int ci = 0; ci < C; ++ci) {
      const M2LEntry& e = t[(size_t)co * C + ci];
      const double ar = e.s1 * G[2 * e.i1] + e.s2 * G[2 * e.i2];
      const double ai = e.s1 * G[2 * e.i1 + 1] + e.s2 * G[2 * e.i2 + 1];
      re += ar * M[2 * ci] - ai * M[2 * ci + 1];
      im += ar * M[2 * ci + 1] + ai * M[2 * ci];
    }
    L[2 * co] = re;
    L[2 * co + 1] = im;
  }
}
}
