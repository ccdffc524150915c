"""Pins of the oracle's solid harmonics (App. A.1, A.2, A.6, A.7) to facts
outside the oracle: the paper's printed table, scipy / sympy Legendre
functions, the Laplace equation, the ladder-operator relations and the
octant symmetries."""
import math
import os

import numpy as np
import pytest
from scipy.special import lpmv

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _table():
    rows = []
    with open(os.path.join(GOLD, "rs_table.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows.append((int(parts[0]), int(parts[1]), parts[2], parts[3]))
    return rows


POINTS = [(0.3, -0.2, 0.5), (-0.7, 0.1, -0.25), (0.05, 0.9, 0.4), (1.3, -1.1, 0.2), (0.0, 0.0, 0.8)]


@pytest.mark.parametrize("pt", POINTS)
def test_table_RSlm(pt):
    """App. A.1, table tab:RSlm: R and S for l <= 2 in Cartesian form."""
    x, y, z = pt
    r = math.sqrt(x * x + y * y + z * z)
    R = oracle.solid_R(2, pt)
    S = oracle.solid_S(2, pt)
    for l, m, er, es in _table():
        pm = 1 if m >= 0 else -1
        env = {"x": x, "y": y, "z": z, "r": r, "pm": pm}
        assert abs(R[oracle.hidx(l, m)] - complex(eval(er, {}, env))) < 1e-14
        assert abs(S[oracle.hidx(l, m)] - complex(eval(es, {}, env))) < 1e-13 * max(1.0, abs(complex(eval(es, {}, env))))


def test_legendre_vs_scipy():
    """App. A.1 definition includes (-1)^m (the Condon-Shortley phase), as scipy's lpmv."""
    for x in [-0.93, -0.4, 0.0, 0.27, 0.81, 0.999]:
        P = oracle.legendre(20, x)
        for l in range(21):
            for m in range(l + 1):
                ref = lpmv(m, l, x)
                assert abs(P[oracle.hidx(l, m)] - ref) <= 1e-12 * max(1.0, abs(ref)), (l, m, x)


def test_legendre_vs_sympy_exact():
    """Rodrigues-form definition of App. A.1, evaluated exactly by sympy at rational x."""
    sympy = pytest.importorskip("sympy")
    X = sympy.Symbol("X")
    for xv in [sympy.Rational(1, 3), sympy.Rational(-5, 7)]:
        s = sympy.sqrt(1 - xv ** 2)
        P = oracle.legendre(8, float(xv), float(s))
        for l in range(9):
            for m in range(l + 1):
                expr = (-s) ** m / (2 ** l * sympy.factorial(l)) * sympy.diff((X ** 2 - 1) ** l, X, l + m)
                ref = float(expr.subs(X, xv))
                assert abs(P[oracle.hidx(l, m)] - ref) <= 1e-12 * max(1.0, abs(ref)), (l, m)


def _fd_grad(f, r, h=1e-5):
    r = np.asarray(r, dtype=float)
    out = []
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        out.append((f(r + e) - f(r - e)) / (2 * h))
    return out


@pytest.mark.parametrize("pt", POINTS[:4])
def test_ladder_operators(pt):
    """App. A.2: d+ R_l^m = R_{l-1}^{m+1}, dz R_l^m = R_{l-1}^m, d- R_l^m = R_{l-1}^{m-1};
    the same for S with l+1.  (d+ = dx + i dy, d- = -dx + i dy.)"""
    p = 6
    R = oracle.solid_R(p, pt)
    S = oracle.solid_S(p + 1, pt)
    gR = _fd_grad(lambda r: oracle.solid_R(p, r), pt, 1e-6)
    gS = _fd_grad(lambda r: oracle.solid_S(p + 1, r), pt, 1e-6)
    for l in range(1, p + 1):
        for m in range(-l, l + 1):
            k = oracle.hidx(l, m)
            dplus = gR[0][k] + 1j * gR[1][k]
            dminus = -gR[0][k] + 1j * gR[1][k]
            dz = gR[2][k]
            tgt = lambda mm: R[oracle.hidx(l - 1, mm)] if abs(mm) <= l - 1 else 0.0
            assert abs(dplus - tgt(m + 1)) < 1e-7 * max(1, abs(R).max())
            assert abs(dminus - tgt(m - 1)) < 1e-7 * max(1, abs(R).max())
            assert abs(dz - tgt(m)) < 1e-7 * max(1, abs(R).max())
    for l in range(0, p):
        for m in range(-l, l + 1):
            k = oracle.hidx(l, m)
            dplus = gS[0][k] + 1j * gS[1][k]
            dminus = -gS[0][k] + 1j * gS[1][k]
            dz = gS[2][k]
            sc = max(1.0, abs(S[oracle.hidx(l + 1, 0)]))
            assert abs(dplus - S[oracle.hidx(l + 1, m + 1)]) < 1e-6 * sc * 10
            assert abs(dminus - S[oracle.hidx(l + 1, m - 1)]) < 1e-6 * sc * 10
            assert abs(dz - S[oracle.hidx(l + 1, m)]) < 1e-6 * sc * 10


def test_laplace():
    """R and S solve the Laplace equation (App. A.1)."""
    pt = np.array([0.4, -0.3, 0.55])
    h = 1e-3
    p = 6

    def lap(f):
        acc = -6 * f(pt)
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            acc = acc + f(pt + e) + f(pt - e)
        return acc / (h * h)

    LR = lap(lambda r: oracle.solid_R(p, r))
    LS = lap(lambda r: oracle.solid_S(p, r))
    S = oracle.solid_S(p, pt)
    assert np.abs(LR).max() < 1e-4
    assert np.abs(LS).max() < 1e-4 * np.abs(S).max() * 100


def test_conjugate_and_octant_symmetries():
    """R_l^{-m} = (-1)^m conj R_l^m (App. A.1), and the octant relation of App. A.6:
    Q(-x, y, -z) = (-1)^l Q(x, -y, z) with Q_l^m = (l+m)! R_l^m."""
    p = 9
    x, y, z = 0.31, -0.47, 0.22
    R = oracle.solid_R(p, (x, y, z))
    Rm = oracle.solid_R(p, (x, -y, z))
    Rf = oracle.solid_R(p, (-x, y, -z))
    for l in range(p + 1):
        for m in range(1, l + 1):
            assert abs(R[oracle.hidx(l, -m)] - (-1) ** m * np.conj(R[oracle.hidx(l, m)])) < 1e-15
        for m in range(0, l + 1):
            assert abs(Rf[oracle.hidx(l, m)] - (-1) ** l * Rm[oracle.hidx(l, m)]) < 1e-14


def test_S_from_Q_relation():
    """App. A.6: S_l^{-m}(x,y,z) = (l-m)! / r^{2l+1} Q_l^m(-x, y, -z), Q_l^m = (l+m)! R_l^m."""
    p = 8
    v = np.array([0.6, 0.25, -0.4])
    r = np.linalg.norm(v)
    S = oracle.solid_S(p, v)
    R = oracle.solid_R(p, (-v[0], v[1], -v[2]))
    for l in range(p + 1):
        for m in range(0, l + 1):
            Q = math.factorial(l + m) * R[oracle.hidx(l, m)]
            ref = math.factorial(l - m) / r ** (2 * l + 1) * Q
            assert abs(S[oracle.hidx(l, -m)] - ref) < 1e-12 * max(1.0, abs(ref))


def test_real_storage_format():
    """App. A.7: X_{l(l+1)+m} = Re X_l^|m| for m >= 0, Im X_l^|m| for m < 0."""
    R = oracle.solid_R(3, (0.1, 0.2, 0.3))
    X = oracle.to_real_storage(R)
    assert X[oracle.hidx(2, 1)] == R[oracle.hidx(2, 1)].real
    assert X[oracle.hidx(2, -1)] == R[oracle.hidx(2, 1)].imag
    assert X[oracle.hidx(3, -3)] == R[oracle.hidx(3, 3)].imag
