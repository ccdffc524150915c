"""The M2L of one cell pair as a two-dimensional cyclic convolution over (order,
degree) indices (Sec. 5, "Another use of FFT convolution", Fig. convmtol): with
f(x, y) = S_{2p-x}^{y} (x = 0..2p, |y| <= 2p - x) and g(x, y) = M_x^y, the cyclic
convolution h = f * g on an NX x NY grid (NX >= 2p+1, NY >= 4p+1, degrees taken
modulo NY) gives L_l^m = h(2p - l, -m).  Checked against the oracle's direct
M2L (Eq. M2L) with numpy FFTs (FP64) at the minimal grid and at the power-of-two
one.  Through p = 7 the two agree to rounding; at p = 12 the FFT mixes terms whose
magnitudes span many decades (S_j grows like j!/r^(j+1)), and the small low-order
locals lose digits: 1e-6 of the largest local, i.e. ~1e-8 relative to the output,
without a per-order rescaling of the grids.  The GPU path keeps the real-matrix
form of App. A.8, which has neither the precision loss nor more flops than this
form up to p = 12."""
import numpy as np
import pytest

import oracle
import synth


def _grid_m2l(p, M, S, NX, NY):
    f = np.zeros((NX, NY), complex)
    g = np.zeros((NX, NY), complex)
    for x in range(2 * p + 1):
        j = 2 * p - x
        for y in range(-j, j + 1):
            f[x, y % NY] = S[oracle.hidx(j, y)]
    for lam in range(p + 1):
        for mu in range(-lam, lam + 1):
            g[lam, mu % NY] = M[oracle.hidx(lam, mu)]
    h = np.fft.ifft2(np.fft.fft2(f) * np.fft.fft2(g))
    L = np.zeros(oracle.nterms(p), complex)
    for l in range(p + 1):
        for m in range(-l, l + 1):
            L[oracle.hidx(l, m)] = h[2 * p - l, (-m) % NY]
    return L


@pytest.mark.parametrize("p,tol", [(0, 1e-12), (1, 1e-12), (2, 1e-12), (5, 1e-12), (7, 1e-12), (12, 1e-7)])
def test_convolution_form_equals_direct_m2l(p, tol):
    g = synth.rng(900 + p)
    # multipoles of a few charges in a cell, translated over a far offset
    pos = g.random((6, 3)) - 0.5
    q = g.standard_normal(6)
    M = oracle.p2m(p, pos, q, (0.0, 0.0, 0.0))
    d = np.array([2.6, -1.3, 3.1])
    S = oracle.solid_S(2 * p, d)
    ref = oracle.m2l(p, M, d)
    NXp = 1 << (2 * p).bit_length()
    NYp = 1 << (4 * p).bit_length()
    for NX, NY in ((2 * p + 1, 4 * p + 1), (NXp, NYp)):
        L = _grid_m2l(p, M, S, NX, NY)
        assert np.abs(L - ref).max() <= tol * np.abs(ref).max(), (NX, NY)


def test_smaller_degree_grid_aliases():
    """NY = 4p (one row short) folds degree 2p onto -2p: the result changes."""
    p = 3
    g = synth.rng(950)
    M = oracle.p2m(p, g.random((5, 3)) - 0.5, g.standard_normal(5), (0.0, 0.0, 0.0))
    d = np.array([2.2, 1.7, -2.9])
    S = oracle.solid_S(2 * p, d)
    ref = oracle.m2l(p, M, d)
    L = _grid_m2l(p, M, S, 2 * p + 1, 4 * p)
    assert np.abs(L - ref).max() > 1e-6 * np.abs(ref).max()
