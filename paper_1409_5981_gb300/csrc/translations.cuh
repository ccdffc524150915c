// Per-element translations of the PMMM path, for registers:
//   * M2L of one wavevector in the real-matrix form of App. A.8 (Eq. realmatrix),
//     applied to Fourier spectra of the real storage channels (Sec. 2.1: the
//     convolution theorem turns the cell sum of Eq. pmmm into one M2L per k);
//   * L2P (Eq. L2P) and the gradient from the order-one L2L (Eq. L2L, Eq. phigrad).
#pragma once
#include "common.cuh"

namespace pmmm {

// Spectrum of the real field Re S_j^kap (re = true) or Im S_j^kap, for any sign of
// kap, from the spectra of the stored components sre[a] = X[sidx(j, a)] and
// sim[a] = X[sidx(j, -a)] (a >= 0), using S_j^{-a} = (-1)^a conj(S_j^a) (App. A.1).
template <typename T, int KAP>
PMMM_HD cpx<T> s_re(const cpx<T>* sre, const cpx<T>* sim) {
  (void)sim;
  if (KAP >= 0) return sre[KAP];
  return ((-KAP) & 1) ? mk(-sre[-KAP].x, -sre[-KAP].y) : sre[-KAP];
}
template <typename T, int KAP>
PMMM_HD cpx<T> s_im(const cpx<T>* sre, const cpx<T>* sim) {
  (void)sre;
  if (KAP == 0) return mk(T(0), T(0));
  if (KAP > 0) return sim[KAP];
  return ((-KAP) & 1) ? sim[-KAP] : mk(-sim[-KAP].x, -sim[-KAP].y);
}

// One term (m, mu) of the real-matrix M2L (Eq. realmatrix) for the current
// output order l and source order lam: the orders m, mu are template constants,
// so that every register array index and sign is fixed at compile time.
template <int P, typename T, int M, int MU>
PMMM_HD void m2l_term(const cpx<T>* sre, const cpx<T>* sim, const cpx<T>* mre, const cpx<T>* mim, cpx<T>* Lre,
                      cpx<T>* Lim) {
  // G^{m,mu} = S_{l+lam}^{-(m+mu)}:  A = Re, B = Im  (Eq. realmatrix)
  const cpx<T> A = s_re<T, -(M + MU)>(sre, sim);
  const cpx<T> B = s_im<T, -(M + MU)>(sre, sim);
  if constexpr (MU == 0) {
    cmac(Lre[M], A, mre[0]);
    cmac(Lim[M], B, mre[0]);
  } else {
    // (-1)^mu G^{m,-mu} = (-1)^mu S_{l+lam}^{-(m-mu)}:  C = Re, D = Im
    cpx<T> C = s_re<T, MU - M>(sre, sim);
    cpx<T> D = s_im<T, MU - M>(sre, sim);
    if constexpr (MU & 1) {
      C = mk(-C.x, -C.y);
      D = mk(-D.x, -D.y);
    }
    // Re L += (A + C) Re M - (B - D) Im M ;  Im L += (B + D) Re M + (A - C) Im M
    cmac(Lre[M], A + C, mre[MU]);
    cmac(Lre[M], D - B, mim[MU]);
    cmac(Lim[M], B + D, mre[MU]);
    cmac(Lim[M], A - C, mim[MU]);
  }
}

// The terms of one source order lam, column by column (mu = 0 .. lam), each
// column over the rows m = 0 .. l.  Both walks stop at their first term outside
// the triangle (mu > lam, m > l): lam and l are the same for every thread of a
// block, so what is left of the walk is skipped by one uniform branch instead of
// being issued under a false predicate.  Each output accumulates its terms in
// the order mu = 0, 1, ... as in a row-by-row walk.
template <int P, typename T, int M, int MU>
struct M2LCol {
  PMMM_HD static void apply(int l, const cpx<T>* sre, const cpx<T>* sim, const cpx<T>* mre, const cpx<T>* mim,
                            cpx<T>* Lre, cpx<T>* Lim) {
    if (M > l) return;
    m2l_term<P, T, M, MU>(sre, sim, mre, mim, Lre, Lim);
    if constexpr (M < P) M2LCol<P, T, M + 1, MU>::apply(l, sre, sim, mre, mim, Lre, Lim);
  }
};
template <int P, typename T, int MU>
struct M2LCols {
  PMMM_HD static void apply(int l, int lam, const cpx<T>* sre, const cpx<T>* sim, const cpx<T>* mre,
                            const cpx<T>* mim, cpx<T>* Lre, cpx<T>* Lim) {
    if (MU > lam) return;
    M2LCol<P, T, 0, MU>::apply(l, sre, sim, mre, mim, Lre, Lim);
    if constexpr (MU < P) M2LCols<P, T, MU + 1>::apply(l, lam, sre, sim, mre, mim, Lre, Lim);
  }
};

// The same walk with the output order L known at compile time (the rows m <= L
// are resolved by the compiler; the source order lam stays a runtime loop, which
// keeps the register arrays of one lam live at a time).
template <int P, int L, typename T, int M, int MU>
struct M2LColL {
  PMMM_HD static void apply(const cpx<T>* sre, const cpx<T>* sim, const cpx<T>* mre, const cpx<T>* mim, cpx<T>* Lre,
                            cpx<T>* Lim) {
    m2l_term<P, T, M, MU>(sre, sim, mre, mim, Lre, Lim);
    if constexpr (M < L) M2LColL<P, L, T, M + 1, MU>::apply(sre, sim, mre, mim, Lre, Lim);
  }
};
template <int P, int L, typename T, int MU>
struct M2LColsL {
  PMMM_HD static void apply(int lam, const cpx<T>* sre, const cpx<T>* sim, const cpx<T>* mre, const cpx<T>* mim,
                            cpx<T>* Lre, cpx<T>* Lim) {
    if (MU > lam) return;
    M2LColL<P, L, T, 0, MU>::apply(sre, sim, mre, mim, Lre, Lim);
    if constexpr (MU < P) M2LColsL<P, L, T, MU + 1>::apply(lam, sre, sim, mre, mim, Lre, Lim);
  }
};
template <int P, int L, typename T, class LM, class LG, class ST>
PMMM_HD void m2l_order_l(int p, LM&& Mk, LG&& Gk, ST&& St) {
  cpx<T> Lre[L + 1], Lim[L + 1];
#pragma unroll
  for (int m = 0; m <= L; ++m) {
    Lre[m] = mk(T(0), T(0));
    Lim[m] = mk(T(0), T(0));
  }
  for (int lam = 0; lam <= p; ++lam) {
    const int j = L + lam;
    cpx<T> mre[P + 1], mim[P + 1];
#pragma unroll
    for (int mu = 0; mu <= P; ++mu) {
      mre[mu] = mk(T(0), T(0));
      mim[mu] = mk(T(0), T(0));
      if (mu <= lam) {
        mre[mu] = Mk(sidx(lam, mu));
        if (mu > 0) mim[mu] = Mk(sidx(lam, -mu));
      }
    }
    cpx<T> sre[L + P + 1], sim[L + P + 1];
#pragma unroll
    for (int a = 0; a <= L + P; ++a) {
      sre[a] = mk(T(0), T(0));
      sim[a] = mk(T(0), T(0));
      if (a <= j) {
        sre[a] = Gk(sidx(j, a));
        if (a > 0) sim[a] = Gk(sidx(j, -a));
      }
    }
    M2LColsL<P, L, T, 0>::apply(lam, sre, sim, mre, mim, Lre, Lim);
  }
#pragma unroll
  for (int m = 0; m <= L; ++m) {
    St(sidx(L, m), Lre[m]);
    if (m > 0) St(sidx(L, -m), Lim[m]);
  }
}

// One output order l of the M2L at one wavevector.
//   Mk(c)  -> spectrum of real channel c of M at this k      (c < (p+1)^2)
//   Gk(s)  -> spectrum of real component s of the kernel      (s < (2p+1)^2)
//   St(c, v) stores the spectrum of real channel c of L.
// The kernel component s = sidx(j, kap) is the real storage of S_j (App. A.7).
template <int P, typename T, class LM, class LG, class ST>
PMMM_HD void m2l_order(int l, int p, LM&& Mk, LG&& Gk, ST&& St) {
  cpx<T> Lre[P + 1], Lim[P + 1];
#pragma unroll
  for (int m = 0; m <= P; ++m) {
    Lre[m] = mk(T(0), T(0));
    Lim[m] = mk(T(0), T(0));
  }
  for (int lam = 0; lam <= p; ++lam) {
    const int j = l + lam;
    cpx<T> mre[P + 1], mim[P + 1];
#pragma unroll
    for (int mu = 0; mu <= P; ++mu) {
      mre[mu] = mk(T(0), T(0));
      mim[mu] = mk(T(0), T(0));
      if (mu <= lam) {
        mre[mu] = Mk(sidx(lam, mu));
        if (mu > 0) mim[mu] = Mk(sidx(lam, -mu));
      }
    }
    cpx<T> sre[2 * P + 1], sim[2 * P + 1];
#pragma unroll
    for (int a = 0; a <= 2 * P; ++a) {
      sre[a] = mk(T(0), T(0));
      sim[a] = mk(T(0), T(0));
      if (a <= j) {
        sre[a] = Gk(sidx(j, a));
        if (a > 0) sim[a] = Gk(sidx(j, -a));
      }
    }
    M2LCols<P, T, 0>::apply(l, lam, sre, sim, mre, mim, Lre, Lim);
  }
#pragma unroll
  for (int m = 0; m <= P; ++m) {
    if (m <= l) {
      St(sidx(l, m), Lre[m]);
      if (m > 0) St(sidx(l, -m), Lim[m]);
    }
  }
}

// ---------------------------------------------------------------------------
// The same M2L with the parity of the kernel spectra used.  Every stored kernel
// component of order j is a real function of the cell offset with
// G(-d) = (-1)^j G(d) (the solid harmonic S_j is homogeneous of parity (-1)^j,
// and the masks, the zero padding and the periodic image sums are symmetric), so
// its spectrum is real for even j and imaginary for odd j.  Gr(s) returns that
// one real number of component s (Re for even j, Im for odd j).  Each
// kernel-spectrum factor of a term is then a real scalar times eps_j (1 or i), and
// eps_j is applied to the moment spectra once per source order (M' = eps_j M): a
// complex product becomes a real scalar times a complex number, half the
// multiply-adds of the complex form, with the kernel spectra half the size.
template <typename T, int KAP>
PMMM_HD T s_re_r(const T* sre, const T* sim) {
  (void)sim;
  if (KAP >= 0) return sre[KAP];
  return ((-KAP) & 1) ? -sre[-KAP] : sre[-KAP];
}
template <typename T, int KAP>
PMMM_HD T s_im_r(const T* sre, const T* sim) {
  (void)sre;
  if (KAP == 0) return T(0);
  if (KAP > 0) return sim[KAP];
  return ((-KAP) & 1) ? sim[-KAP] : -sim[-KAP];
}
// a += s v, s real: two multiply-adds
template <typename T>
PMMM_HD void rmac(cpx<T>& a, T s, cpx<T> v) {
  a.x = fma(s, v.x, a.x);
  a.y = fma(s, v.y, a.y);
}

// Term (m, mu) of Eq. realmatrix with real kernel scalars and M' = eps_j M.
template <int P, typename T, int M, int MU>
PMMM_HD void m2l_term_par(const T* sre, const T* sim, const cpx<T>* mre, const cpx<T>* mim, cpx<T>* Lre,
                          cpx<T>* Lim) {
  const T A = s_re_r<T, -(M + MU)>(sre, sim);
  const T B = s_im_r<T, -(M + MU)>(sre, sim);
  if constexpr (MU == 0) {
    rmac(Lre[M], A, mre[0]);
    if constexpr (M != 0) rmac(Lim[M], B, mre[0]);
  } else {
    T C = s_re_r<T, MU - M>(sre, sim);
    T D = s_im_r<T, MU - M>(sre, sim);
    if constexpr (MU & 1) {
      C = -C;
      D = -D;
    }
    rmac(Lre[M], A + C, mre[MU]);
    rmac(Lre[M], D - B, mim[MU]);
    rmac(Lim[M], B + D, mre[MU]);
    rmac(Lim[M], A - C, mim[MU]);
  }
}

template <int P, typename T, int M, int MU>
struct M2LColPar {
  PMMM_HD static void apply(int l, const T* sre, const T* sim, const cpx<T>* mre, const cpx<T>* mim, cpx<T>* Lre,
                            cpx<T>* Lim) {
    if (M > l) return;
    m2l_term_par<P, T, M, MU>(sre, sim, mre, mim, Lre, Lim);
    if constexpr (M < P) M2LColPar<P, T, M + 1, MU>::apply(l, sre, sim, mre, mim, Lre, Lim);
  }
};
template <int P, typename T, int MU>
struct M2LColsPar {
  PMMM_HD static void apply(int l, int lam, const T* sre, const T* sim, const cpx<T>* mre, const cpx<T>* mim,
                            cpx<T>* Lre, cpx<T>* Lim) {
    if (MU > lam) return;
    M2LColPar<P, T, 0, MU>::apply(l, sre, sim, mre, mim, Lre, Lim);
    if constexpr (MU < P) M2LColsPar<P, T, MU + 1>::apply(l, lam, sre, sim, mre, mim, Lre, Lim);
  }
};

// One output order l of the M2L at one wavevector from the parity-reduced kernel
// spectra: Mk(c) as in m2l_order, Gr(s) the real number of component s, St(c, v).
template <int P, typename T, class LM, class LG, class ST>
PMMM_HD void m2l_order_par(int l, int p, LM&& Mk, LG&& Gr, ST&& St) {
  cpx<T> Lre[P + 1], Lim[P + 1];
#pragma unroll
  for (int m = 0; m <= P; ++m) {
    Lre[m] = mk(T(0), T(0));
    Lim[m] = mk(T(0), T(0));
  }
  for (int lam = 0; lam <= p; ++lam) {
    const int j = l + lam;
    const bool odd = (j & 1) != 0;
    cpx<T> mre[P + 1], mim[P + 1];
#pragma unroll
    for (int mu = 0; mu <= P; ++mu) {
      if (mu <= lam) {
        cpx<T> v = Mk(sidx(lam, mu));
        mre[mu] = odd ? mk(-v.y, v.x) : v;
        if (mu > 0) {
          v = Mk(sidx(lam, -mu));
          mim[mu] = odd ? mk(-v.y, v.x) : v;
        }
      }
    }
    T sre[2 * P + 1], sim[2 * P + 1];
#pragma unroll
    for (int a = 0; a <= 2 * P; ++a) {
      if (a <= j) {
        sre[a] = Gr(sidx(j, a));
        if (a > 0) sim[a] = Gr(sidx(j, -a));
      }
    }
    M2LColsPar<P, T, 0>::apply(l, lam, sre, sim, mre, mim, Lre, Lim);
  }
#pragma unroll
  for (int m = 0; m <= P; ++m) {
    if (m <= l) {
      St(sidx(l, m), Lre[m]);
      if (m > 0) St(sidx(l, -m), Lim[m]);
    }
  }
}

// L2P of Eq. L2P and the gradient through the order-one L2L of Eq. L2L
// (Eq. phigrad: dPhi/dx = -Re L'_1^1, dPhi/dy = Im L'_1^1, dPhi/dz = L'_1^0).
//   L(c) -> real channel c of the local expansion; R: real storage of R(r - r_L).
template <int P, typename T, class LL>
PMMM_HD void l2p_real(LL&& Lc, const T* R, T& phi, T& gx, T& gy, T& gz) {
  T f = T(0), l10 = T(0), l11r = T(0), l11i = T(0);
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    // Phi = sum_l [L_l^0 R_l^0 + 2 sum_{m>0} Re(L_l^m R_l^m)]
    const T L0 = Lc(sidx(l, 0));
    f += L0 * R[sidx(l, 0)];
#pragma unroll
    for (int m = 1; m <= l; ++m) {
      const T lr = Lc(sidx(l, m)), li = Lc(sidx(l, -m));
      f += T(2) * (lr * R[sidx(l, m)] - li * R[sidx(l, -m)]);
    }
    if (l >= 1) {
      // L'_1^0 = sum_l [L_l^0 R_{l-1}^0 + 2 sum_{mu=1}^{l-1} Re(L_l^mu R_{l-1}^mu)]
      l10 += L0 * R[sidx(l - 1, 0)];
#pragma unroll
      for (int m = 1; m <= l - 1; ++m) {
        const T lr = Lc(sidx(l, m)), li = Lc(sidx(l, -m));
        l10 += T(2) * (lr * R[sidx(l - 1, m)] - li * R[sidx(l - 1, -m)]);
      }
      // L'_1^1 = sum_l [ sum_{mu=1}^{l} L_l^mu R_{l-1}^{mu-1}
      //                  - sum_{nu=0}^{l-2} conj(L_l^nu R_{l-1}^{nu+1}) ]
#pragma unroll
      for (int m = 1; m <= l; ++m) {
        const T lr = Lc(sidx(l, m)), li = Lc(sidx(l, -m));
        const T rr = R[sidx(l - 1, m - 1)], ri = (m - 1 > 0) ? R[sidx(l - 1, -(m - 1))] : T(0);
        l11r += lr * rr - li * ri;
        l11i += lr * ri + li * rr;
      }
#pragma unroll
      for (int nu = 0; nu <= l - 2; ++nu) {
        const T lr = Lc(sidx(l, nu)), li = (nu > 0) ? Lc(sidx(l, -nu)) : T(0);
        const T rr = R[sidx(l - 1, nu + 1)], ri = R[sidx(l - 1, -(nu + 1))];
        // -conj(a b) = -(Re(ab)) + i Im(ab)
        l11r -= lr * rr - li * ri;
        l11i += lr * ri + li * rr;
      }
    }
  }
  phi = f;
  gx = -l11r;
  gy = l11i;
  gz = l10;
}

// L2P and its gradient (same sums as l2p_real) with the regular harmonics of
// r - r_L computed on the fly column by column (recurrences of App. A.6): only
// the current column R_l^m and the previous one R_l^{m-1} are kept, so the
// register count grows as O(P) instead of O(P^2).  At column m, row l:
//   potential      L_l^m R_l^m
//   L'_1^0 term    L_l^m R_{l-1}^m                        (m <= l-1)
//   L'_1^1 terms   L_l^m R_{l-1}^{m-1}                    (m >= 1)
//                  -conj(L_l^{m-1} R_{l-1}^m)             (m >= 1, l >= m+1)
template <int P, typename T, class LL>
PMMM_HD void l2p_stream(LL&& Lc, T x, T y, T z, T& phi, T& gx, T& gy, T& gz) {
  const T r2 = x * x + y * y + z * z;
  T pr[P + 1], pi[P + 1], cr[P + 1], ci[P + 1];
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    pr[l] = pi[l] = cr[l] = ci[l] = T(0);
  }
  T f = T(0), l10 = T(0), l11r = T(0), l11i = T(0);
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
#pragma unroll
    for (int l = m; l <= P; ++l) {
      T rr, ri;
      if (l == m) {
        rr = mmr;
        ri = mmi;
      } else if (l == m + 1) {
        rr = z * cr[l - 1];
        ri = z * ci[l - 1];
      } else {
        const T c1 = T(2 * l - 1) / T((l - m) * (l + m));
        const T c2 = T(1) / T((l - m) * (l + m));
        rr = c1 * z * cr[l - 1] - c2 * r2 * cr[l - 2];
        ri = c1 * z * ci[l - 1] - c2 * r2 * ci[l - 2];
      }
      const T Lr = Lc(sidx(l, m)), Li = (m > 0) ? Lc(sidx(l, -m)) : T(0);
      if (m == 0) {
        f += Lr * rr;
        if (l >= 1) l10 += Lr * cr[l - 1];
      } else {
        f += T(2) * (Lr * rr - Li * ri);
        if (l >= m + 1) l10 += T(2) * (Lr * cr[l - 1] - Li * ci[l - 1]);
        // L_l^m R_{l-1}^{m-1}
        const T qr = pr[l - 1], qi = (m > 1) ? pi[l - 1] : T(0);
        l11r += Lr * qr - Li * qi;
        l11i += Lr * qi + Li * qr;
        if (l >= m + 1) {
          // -conj(L_l^{m-1} R_{l-1}^m)
          const T Mr = Lc(sidx(l, m - 1)), Mi = (m > 1) ? Lc(sidx(l, -(m - 1))) : T(0);
          l11r -= Mr * cr[l - 1] - Mi * ci[l - 1];
          l11i += Mr * ci[l - 1] + Mi * cr[l - 1];
        }
      }
      cr[l] = rr;
      ci[l] = ri;
    }
#pragma unroll
    for (int l = m; l <= P; ++l) {
      pr[l] = cr[l];
      pi[l] = ci[l];
    }
  }
  phi = f;
  gx = -l11r;
  gy = l11i;
  gz = l10;
}

}  // namespace pmmm
