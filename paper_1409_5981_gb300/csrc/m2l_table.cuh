// Entry table of the real-matrix M2L (App. A.8, Eq. realmatrix): every entry of
// the (p+1)^2 x (p+1)^2 real matrix that maps the real storage channels of M to
// those of L is a signed sum of at most two real storage components of the
// kernel S_{l+lam} (App. A.7).  In Fourier space the same combination of the
// component spectra gives the matrix A~(k) of one wavevector (Sec. 2.1), which
// the batched M2L applies to all systems at once.
#pragma once
#include <vector>

#include "common.cuh"

namespace pmmm {

struct M2LEntry {
  int i1, s1, i2, s2;  // component indices and signs (sign 0: term absent)
};

namespace m2ltab {
// Re / Im of S_j^kap in terms of stored components, for any sign of kap
// (S_j^{-a} = (-1)^a conj(S_j^a), App. A.1).
inline void re_s(int j, int kap, int& idx, int& sg) {
  if (kap >= 0) {
    idx = sidx(j, kap);
    sg = 1;
  } else {
    idx = sidx(j, -kap);
    sg = ((-kap) & 1) ? -1 : 1;
  }
}
inline void im_s(int j, int kap, int& idx, int& sg) {
  if (kap == 0) {
    idx = 0;
    sg = 0;
  } else if (kap > 0) {
    idx = sidx(j, -kap);
    sg = 1;
  } else {
    idx = sidx(j, kap);
    sg = ((-kap) & 1) ? 1 : -1;
  }
}
inline void put(std::vector<M2LEntry>& t, int C, int cout, int cin, int i1, int s1, int i2, int s2) {
  M2LEntry& e = t[(size_t)cout * C + cin];
  e.i1 = i1;
  e.s1 = s1;
  e.i2 = i2;
  e.s2 = s2;
}
}  // namespace m2ltab

// tab[c_out * C + c_in], C = (p+1)^2; entry value = s1 * G[i1] + s2 * G[i2].
inline std::vector<M2LEntry> build_m2l_table(int p) {
  using namespace m2ltab;
  const int C = (p + 1) * (p + 1);
  std::vector<M2LEntry> t((size_t)C * C, M2LEntry{0, 0, 0, 0});
  for (int l = 0; l <= p; ++l)
    for (int lam = 0; lam <= p; ++lam) {
      const int j = l + lam;
      for (int m = 0; m <= l; ++m)
        for (int mu = 0; mu <= lam; ++mu) {
          int ai, as, bi, bs;  // A = Re, B = Im of G^{m,mu} = S_j^{-(m+mu)}
          re_s(j, -(m + mu), ai, as);
          im_s(j, -(m + mu), bi, bs);
          const int oRe = sidx(l, m), oIm = sidx(l, -m);
          if (mu == 0) {
            put(t, C, oRe, sidx(lam, 0), ai, as, 0, 0);
            if (m > 0) put(t, C, oIm, sidx(lam, 0), bi, bs, 0, 0);
            continue;
          }
          int ci, cs_, di, ds;  // C = (-1)^mu Re, D = (-1)^mu Im of S_j^{mu-m}
          re_s(j, mu - m, ci, cs_);
          im_s(j, mu - m, di, ds);
          if (mu & 1) {
            cs_ = -cs_;
            ds = -ds;
          }
          const int iRe = sidx(lam, mu), iIm = sidx(lam, -mu);
          // Re L += (A + C) Re M + (D - B) Im M ;  Im L += (B + D) Re M + (A - C) Im M
          put(t, C, oRe, iRe, ai, as, ci, cs_);
          put(t, C, oRe, iIm, di, ds, bi, -bs);
          if (m > 0) {
            put(t, C, oIm, iRe, bi, bs, di, ds);
            put(t, C, oIm, iIm, ai, as, ci, -cs_);
          }
        }
    }
  return t;
}

}  // namespace pmmm
