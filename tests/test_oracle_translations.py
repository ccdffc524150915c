"""Pins of the oracle's translations (App. A.2-A.5) to the addition theorems,
the expansion of 1/r, finite-difference gradients and the error estimate."""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _cluster(n, s, radius):
    g = synth.rng(s)
    pos = (g.random((n, 3)) - 0.5) * 2 * radius / math.sqrt(3)
    q = 2 * g.random(n) - 1
    return pos, q


def test_expansion_of_inverse_distance():
    """Eq. expand: 1/|rS - rR| = sum S_lam^{-mu}(rS) R_lam^mu(-rR) for |rS| > |rR|,
    converging geometrically in (|rR|/|rS|)."""
    rS = np.array([0.9, -0.4, 0.7])
    rR = np.array([0.1, 0.2, -0.15])
    exact = 1.0 / np.linalg.norm(rS - rR)
    ratio = np.linalg.norm(rR) / np.linalg.norm(rS)
    prev = None
    for p in [2, 4, 8, 12, 16]:
        S = oracle.solid_S(p, rS)
        R = oracle.solid_R(p, -rR)
        acc = sum(S[oracle.hidx(l, -m)] * R[oracle.hidx(l, m)] for l in range(p + 1) for m in range(-l, l + 1))
        err = abs(acc - exact)
        assert abs(acc.imag) < 1e-14
        assert err < 4 * ratio ** (p + 1) / (1 - ratio) * exact
        if prev is not None:
            assert err < prev
        prev = err
    assert prev < 1e-12


def test_m2p_converges_to_direct():
    """P2M (Eq. P2M) then M2P (Eq. M2P) approach the direct sum outside the sphere."""
    pos, q = _cluster(40, 11, 0.3)
    tgt = np.array([1.1, 0.4, -0.6])
    exact = float(np.sum(q / np.linalg.norm(tgt - pos, axis=1)))
    errs = []
    for p in [2, 5, 8, 12]:
        M = oracle.p2m(p, pos, q, np.zeros(3))
        errs.append(abs(oracle.m2p(p, M, tgt) - exact))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-7 * np.abs(q).sum()


def test_m2m_exact():
    """Eq. M2M is exact: P2M at centre A, M2M to centre B == P2M at centre B."""
    p = 8
    pos, q = _cluster(25, 12, 0.2)
    A = np.array([0.05, -0.03, 0.02])
    B = np.array([-0.1, 0.2, 0.15])
    MA = oracle.p2m(p, pos, q, A)
    MB = oracle.p2m(p, pos, q, B)
    MAB = oracle.m2m(p, MA, B - A)
    assert np.abs(MAB - MB).max() < 1e-13 * max(1.0, np.abs(MB).max())


def test_l2l_exact_and_l2p():
    """Eq. L2L is exact at full order: L2P after L2L == L2P at the original centre."""
    p = 7
    g = synth.rng(13)
    L = g.standard_normal(oracle.nterms(p)) + 1j * g.standard_normal(oracle.nterms(p))
    # impose the conjugate relation L_l^{-m} = (-1)^m conj L_l^m
    for l in range(p + 1):
        L[oracle.hidx(l, 0)] = L[oracle.hidx(l, 0)].real
        for m in range(1, l + 1):
            L[oracle.hidx(l, -m)] = (-1) ** m * np.conj(L[oracle.hidx(l, m)])
    shift = np.array([0.12, -0.07, 0.05])
    Lp = oracle.l2l(p, p, L, shift)
    r = np.array([0.03, 0.02, -0.04])
    a = oracle.l2p_phi(p, Lp, r)
    b = oracle.l2p_phi(p, L, r + shift)
    assert abs(a - b) < 1e-12 * max(1.0, abs(b))


def test_gradient_from_first_order_local():
    """Eq. phigrad: the order-one L2L gives the gradient of Eq. L2P (finite differences)."""
    p = 6
    g = synth.rng(14)
    L = g.standard_normal(oracle.nterms(p)) + 1j * g.standard_normal(oracle.nterms(p))
    for l in range(p + 1):
        L[oracle.hidx(l, 0)] = L[oracle.hidx(l, 0)].real
        for m in range(1, l + 1):
            L[oracle.hidx(l, -m)] = (-1) ** m * np.conj(L[oracle.hidx(l, m)])
    r = np.array([0.21, -0.13, 0.09])
    phi, grad = oracle.l2p(p, L, r)
    assert abs(phi - oracle.l2p_phi(p, L, r)) < 1e-13
    h = 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (oracle.l2p_phi(p, L, r + e) - oracle.l2p_phi(p, L, r - e)) / (2 * h)
        assert abs(fd - grad[a]) < 1e-7


def test_m2l_converges_and_gradient():
    """P2M -> M2L (Eq. M2L) -> L2P approaches the direct potential and force of a
    distant cluster; the error falls with p."""
    src, q = _cluster(30, 15, 0.25)
    trg = np.array([[0.05, -0.1, 0.08], [-0.12, 0.03, 0.1]])
    cL = np.array([1.3, 0.2, -0.4])
    exact_phi = np.array([np.sum(q / np.linalg.norm(cL + t - src, axis=1)) for t in trg])
    exact_g = np.array([-np.sum(q[:, None] * (cL + t - src) / np.linalg.norm(cL + t - src, axis=1)[:, None] ** 3, axis=0) for t in trg])
    errs = []
    for p in [2, 4, 6, 9]:
        M = oracle.p2m(p, src, q, np.zeros(3))
        L = oracle.m2l(p, M, cL)
        e = 0
        for t, ph, gr in zip(trg, exact_phi, exact_g):
            f, g = oracle.l2p(p, L, t)
            e = max(e, abs(f - ph), np.abs(g - gr).max())
        errs.append(e)
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-5


def test_error_estimate_factors():
    """Eq. errest and the per-order factors printed after it (0.76, 0.41, 0.28, 0.21)."""
    with open(os.path.join(GOLD, "errest.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for c, printed in rows:
        c = int(c)
        factor = oracle.error_estimate(c, 1) / oracle.error_estimate(c, 0)
        assert round(factor, 2) == float(printed)


def test_incomplete_gamma_vs_scipy():
    """App. B.1 split functions Gamma(l+1/2, x)/Gamma(l+1/2) and gamma(l+1/2, x)/Gamma(l+1/2)."""
    from scipy.special import gammainc, gammaincc
    for l in range(0, 26):
        for x in [1e-6, 1e-3, 0.05, 0.7, 2.0, 5.5, 12.0, 30.0, 60.0]:
            q = oracle.gammaQ_half(l, x)
            p = oracle.gammaP_half(l, x)
            rq, rp = gammaincc(l + 0.5, x), gammainc(l + 0.5, x)
            assert abs(q - rq) <= 1e-13 * max(rq, 1e-300) + 1e-300 or abs(q - rq) < 1e-15, (l, x, q, rq)
            assert abs(p - rp) <= 1e-12 * rp + 1e-300, (l, x, p, rp)
