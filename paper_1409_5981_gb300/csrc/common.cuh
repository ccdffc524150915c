// Shared device/host helpers of the PMMM GPU library: complex type, the real
// storage index of App. A.7, and a host/device function qualifier that lets
// the per-element math be compiled by a host compiler for unit tests.
#pragma once
#include <stdint.h>
#include <math.h>

#if defined(__CUDACC__)
#define PMMM_HD __host__ __device__ __forceinline__
#define PMMM_DEV __device__ __forceinline__
#else
#define PMMM_HD inline
#define PMMM_DEV inline
#endif

#ifndef PMMM_PMAX
#define PMMM_PMAX 12  // highest expansion order with compiled kernels
#endif

namespace pmmm {

template <typename T>
struct alignas(2 * sizeof(T)) cpx {
  T x, y;  // real, imaginary
};

template <typename T> PMMM_HD cpx<T> mk(T a, T b) { cpx<T> r; r.x = a; r.y = b; return r; }
template <typename T> PMMM_HD cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T> PMMM_HD cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T> PMMM_HD cpx<T> operator*(cpx<T> a, cpx<T> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> PMMM_HD cpx<T> operator*(T s, cpx<T> a) { return mk(s * a.x, s * a.y); }
template <typename T> PMMM_HD cpx<T> conjg(cpx<T> a) { return mk(a.x, -a.y); }
// multiply by +i (s = +1) or -i (s = -1)
template <typename T> PMMM_HD cpx<T> mul_si(cpx<T> a, int s) { return s > 0 ? mk(-a.y, a.x) : mk(a.y, -a.x); }
// a += b * c as four fused multiply-adds into the accumulator (one rounding each)
template <typename T> PMMM_HD void cmac(cpx<T>& a, cpx<T> b, cpx<T> c) {
  a.x = fma(b.x, c.x, a.x);
  a.x = fma(-b.y, c.y, a.x);
  a.y = fma(b.x, c.y, a.y);
  a.y = fma(b.y, c.x, a.y);
}

// Real storage index of App. A.7: X[l(l+1)+m] = Re X_l^|m| (m >= 0), Im X_l^|m| (m < 0).
PMMM_HD constexpr int sidx(int l, int m) { return l * (l + 1) + m; }
PMMM_HD constexpr int nterms(int p) { return (p + 1) * (p + 1); }

}  // namespace pmmm
