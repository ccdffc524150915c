"""Pins of the oracle's Green functions.

Open boundary (Sec. 2.1, App. C): S(d h) with the nearest (2c+1)^3 cells masked.
Periodic (App. B, Eqs. infsum, greenPBC): the Ewald-split lattice sum must
  * not depend on alpha (both sums converged);
  * equal a brute-force real-space lattice sum where that sum converges
    absolutely (order j >= 5 here);
  * reduce at l = 0 / l = 1 to the classic Ewald potential / field of a unit
    charge (App. B.2 remark), once the masked image is added back.
"""
import numpy as np
import pytest

import oracle


def test_open_green_mask():
    p, c = 3, 1
    h = (0.25, 0.25, 0.25)
    assert np.all(oracle.green_open(p, c, h, (1, -1, 0)) == 0)
    assert np.all(oracle.green_open(p, 2, h, (2, 0, -2)) == 0)
    G = oracle.green_open(p, c, h, (2, -1, 0))
    ref = oracle.solid_S(2 * p, (0.5, -0.25, 0.0))
    assert np.abs(G - ref).max() == 0.0


@pytest.mark.parametrize("d", [(0, 0, 0), (1, 0, 0), (3, 2, 7), (4, 4, 4), (5, 1, 2)])
def test_periodic_green_alpha_independent(d):
    p, c = 4, 1
    mesh = (8, 8, 8)
    G1 = oracle.green_periodic(p, c, mesh, (1, 1, 1), 1.5, 7, d)
    G2 = oracle.green_periodic(p, c, mesh, (1, 1, 1), 2.3, 7, d)
    # The l = 0 reciprocal sum omits k = 0, so G_0^0 carries the alpha-dependent
    # constant pi/(V alpha^2) (cancelled by Q = 0, or by the charged-system
    # correction).  The self-cell entry also lacks the limit -2 alpha/sqrt(pi) of the
    # masked n = 0 image, which the correction procedure supplies separately.
    for G, a in ((G1, 1.5), (G2, 2.3)):
        G[0] -= np.pi / a ** 2
        if d == (0, 0, 0):
            G[0] -= 2 * a / np.sqrt(np.pi)
    for j in range(2 * p + 1):
        sl = slice(j * j, (j + 1) * (j + 1))
        scale = max(1.0, np.abs(G1[sl]).max())
        assert np.abs(G1[sl] - G2[sl]).max() < 1e-10 * scale, j


def test_periodic_green_vs_bruteforce_lattice_sum():
    """For j >= 5 the lattice sum of S_j converges absolutely; sum images directly."""
    p, c = 4, 1
    mesh = (8, 8, 8)
    d = (3, 1, 6)
    G = oracle.green_periodic(p, c, mesh, (1, 1, 1), 1.5, 7, d)
    dm = np.array([3, 1, -2])  # minimum image of d
    r0 = dm / 8.0
    ref = np.zeros_like(G)
    R = 14
    rng_ = np.arange(-R, R + 1)
    for a in rng_:
        for b in rng_:
            for e in rng_:
                if a * a + b * b + e * e > R * R:
                    continue
                ref += oracle.solid_S(2 * p, r0 + np.array([a, b, e]))
    for j in range(5, 2 * p + 1):
        sl = slice(j * j, (j + 1) * (j + 1))
        scale = np.abs(G[sl]).max()
        assert np.abs(G[sl] - ref[sl]).max() < 2e-8 * scale, j


@pytest.mark.parametrize("d", [(0, 0, 0), (1, 1, 0), (3, 2, 7), (4, 0, 4)])
def test_periodic_green_low_order_is_ewald(d):
    """l = 0: G_0^0 + (masked image 1/r) - pi/(V alpha^2) = Ewald potential at r_d of a
    unit charge at the origin (probe with zero charge); l = 1: the field."""
    p, c = 2, 1
    mesh = (8, 8, 8)
    alpha = 1.5
    G = oracle.green_periodic(p, c, mesh, (1, 1, 1), alpha, 7, d)
    dm = np.array([v if 2 * v <= 8 else v - 8 for v in d])
    rd = dm / 8.0
    near = np.abs(dm).max() <= c
    pos = np.array([[0.0, 0.0, 0.0], rd]) + 0.5
    q = np.array([1.0, 0.0])
    phi, grad = oracle.ewald(pos, q, (1, 1, 1), tol=1e-14)
    V = 1.0
    if d == (0, 0, 0):
        # self cell: Ewald potential of a charge at itself minus 1/r singularity:
        # lim (phi_ewald(r) - 1/r) = G_0^0(0) - 2 alpha/sqrt(pi) - pi/(V alpha^2)
        ph2, _ = oracle.ewald(np.array([[0.5, 0.5, 0.5]]), np.array([1.0]), (1, 1, 1), tol=1e-14)
        # Ewald phi_i of a single charge already subtracts the self term -2 alpha_E/sqrt(pi)
        # and the background; its value is the regular part of the lattice potential.
        assert abs(G[0].real - 2 * alpha / np.sqrt(np.pi) - np.pi / (V * alpha ** 2) - ph2[0]) < 1e-11
        return
    S = oracle.solid_S(1, rd)
    add = S if near else np.zeros_like(S)
    assert abs(G[0].real + add[0].real - np.pi / (V * alpha ** 2) - phi[1]) < 1e-11
    # field: by the ladder relations d+ S_0^0 = S_1^1, d- S_0^0 = S_1^-1,
    # grad (1/r) = (Re S_1^1, Im S_1^1, S_1^0), summed over the images
    gl = np.array([(G[3] + add[3]).real, (G[3] + add[3]).imag, (G[2] + add[2]).real])
    assert np.abs(gl - grad[1]).max() < 1e-10


def test_periodic_green_nmax_convergence():
    p, c = 5, 1
    mesh = (8, 8, 8)
    d = (2, 5, 1)
    Ga = oracle.green_periodic(p, c, mesh, (1, 1, 1), 1.5, 4, d)
    Gb = oracle.green_periodic(p, c, mesh, (1, 1, 1), 1.5, 7, d)
    for j in range(2 * p + 1):
        sl = slice(j * j, (j + 1) * (j + 1))
        assert np.abs(Ga[sl] - Gb[sl]).max() < 1e-12 * max(1.0, np.abs(Gb[sl]).max())
