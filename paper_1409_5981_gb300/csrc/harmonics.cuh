// Solid harmonics by Cartesian recurrences (App. A.6), written for registers.
//
// Regular harmonics, with the 1/(l+m)! factor of the definition (App. A.1)
// folded into the recurrence of the scaled Legendre functions of App. A.6:
//   R_0^0     = 1
//   R_m^m     = -(x + i y) / (2m) * R_{m-1}^{m-1}
//   R_{m+1}^m = z R_m^m
//   R_l^m     = ((2l-1) z R_{l-1}^m - r^2 R_{l-2}^m) / ((l-m)(l+m))      (l >= m+2)
// Singular harmonics (definition of App. A.1, same recurrence in 1/r):
//   S_0^0     = 1/r
//   S_m^m     = -(2m-1) (x + i y) / r^2 * S_{m-1}^{m-1}
//   S_l^m     = -((2l-1) z S_{l-1}^m + (l+m-1)(l-m-1) S_{l-2}^m) / r^2  (l >= m+1)
// Both are stored in the real format of App. A.7.
#pragma once
#include "common.cuh"

namespace pmmm {

// X[sidx(l, m)] = Re R_l^m, X[sidx(l, -m)] = Im R_l^m for 0 <= m <= l <= P.
template <int P, typename T>
PMMM_HD void regular_real(T x, T y, T z, T* X) {
  const T r2 = x * x + y * y + z * z;
  T mmr = T(1), mmi = T(0);  // R_m^m
#pragma unroll
  for (int m = 0; m <= P; ++m) {
    if (m > 0) {
      // R_m^m = -(x + i y)/(2m) R_{m-1}^{m-1}
      const T s = T(-1) / T(2 * m);
      const T nr = s * (x * mmr - y * mmi);
      const T ni = s * (x * mmi + y * mmr);
      mmr = nr;
      mmi = ni;
    }
    X[sidx(m, m)] = mmr;
    if (m > 0) X[sidx(m, -m)] = mmi;
    T ar = mmr, ai = mmi;        // R_{l-2}^m (set at l = m+2)
    T br = T(0), bi = T(0);      // R_{l-1}^m
    if (m + 1 <= P) {
      br = z * mmr;
      bi = z * mmi;
      X[sidx(m + 1, m)] = br;
      if (m > 0) X[sidx(m + 1, -m)] = bi;
    }
#pragma unroll
    for (int l = m + 2; l <= P; ++l) {
      const T c1 = T(2 * l - 1) / T((l - m) * (l + m));
      const T c2 = T(1) / T((l - m) * (l + m));
      const T cr = c1 * z * br - c2 * r2 * ar;
      const T ci = c1 * z * bi - c2 * r2 * ai;
      X[sidx(l, m)] = cr;
      if (m > 0) X[sidx(l, -m)] = ci;
      ar = br; ai = bi;
      br = cr; bi = ci;
    }
  }
}

// The same regular harmonics streamed column by column (m = 0..P, then
// l = m..P) to a callback f(l, m, Re R_l^m, Im R_l^m), keeping only the two
// previous rows of the current column: O(P) registers.
template <int P, typename T, class F>
PMMM_HD void regular_stream(T x, T y, T z, F&& f) {
  const T r2 = x * x + y * y + z * z;
  T mmr = T(1), mmi = T(0);
#pragma unroll
  for (int m = 0; m <= P; ++m) {
    if (m > 0) {
      const T s = T(-1) / T(2 * m);
      const T nr = s * (x * mmr - y * mmi);
      const T ni = s * (x * mmi + y * mmr);
      mmr = nr;
      mmi = ni;
    }
    f(m, m, mmr, mmi);
    T ar = mmr, ai = mmi, br = T(0), bi = T(0);
    if (m + 1 <= P) {
      br = z * mmr;
      bi = z * mmi;
      f(m + 1, m, br, bi);
    }
#pragma unroll
    for (int l = m + 2; l <= P; ++l) {
      const T c1 = T(2 * l - 1) / T((l - m) * (l + m));
      const T c2 = T(1) / T((l - m) * (l + m));
      const T cr = c1 * z * br - c2 * r2 * ar;
      const T ci = c1 * z * bi - c2 * r2 * ai;
      f(l, m, cr, ci);
      ar = br; ai = bi;
      br = cr; bi = ci;
    }
  }
}

// The regular harmonics of regular_real for a runtime order p, handed to a
// callback f(c, value) with c the real storage index of App. A.7 (used for the
// small translation tables built once per plan).
template <typename T, class F>
PMMM_HD void regular_real_rt(int p, T x, T y, T z, F&& f) {
  const T r2 = x * x + y * y + z * z;
  T mmr = T(1), mmi = T(0);
  for (int m = 0; m <= p; ++m) {
    if (m > 0) {
      const T s = T(-1) / T(2 * m);
      const T nr = s * (x * mmr - y * mmi);
      const T ni = s * (x * mmi + y * mmr);
      mmr = nr;
      mmi = ni;
    }
    f(sidx(m, m), mmr);
    if (m > 0) f(sidx(m, -m), mmi);
    T ar = mmr, ai = mmi, br = T(0), bi = T(0);
    if (m + 1 <= p) {
      br = z * mmr;
      bi = z * mmi;
      f(sidx(m + 1, m), br);
      if (m > 0) f(sidx(m + 1, -m), bi);
    }
    for (int l = m + 2; l <= p; ++l) {
      const T c1 = T(2 * l - 1) / T((l - m) * (l + m));
      const T c2 = T(1) / T((l - m) * (l + m));
      const T cr = c1 * z * br - c2 * r2 * ar;
      const T ci = c1 * z * bi - c2 * r2 * ai;
      f(sidx(l, m), cr);
      if (m > 0) f(sidx(l, -m), ci);
      ar = br; ai = bi;
      br = cr; bi = ci;
    }
  }
}

// Singular harmonics S_l^m for one m >= 0 and l = m .. J, handed to a callback
// f(l, Re S_l^m, Im S_l^m).  Runtime orders (used by the Green function set-up).
template <typename T, typename F>
PMMM_HD void singular_column(int m, int J, T x, T y, T z, F&& f) {
  const T r2 = x * x + y * y + z * z;
  const T ir2 = T(1) / r2;
  T sr = T(1) / sqrt(r2), si = T(0);  // S_0^0
  for (int k = 1; k <= m; ++k) {
    const T s = -T(2 * k - 1) * ir2;
    const T nr = s * (x * sr - y * si);
    const T ni = s * (x * si + y * sr);
    sr = nr;
    si = ni;
  }
  f(m, sr, si);
  T ar = T(0), ai = T(0);  // S_{l-2}^m
  T br = sr, bi = si;      // S_{l-1}^m
  for (int l = m + 1; l <= J; ++l) {
    const T c1 = T(2 * l - 1);
    const T c2 = T((l + m - 1) * (l - m - 1));
    const T cr = -(c1 * z * br + c2 * ar) * ir2;
    const T ci = -(c1 * z * bi + c2 * ai) * ir2;
    f(l, cr, ci);
    ar = br; ai = bi;
    br = cr; bi = ci;
  }
}

}  // namespace pmmm
