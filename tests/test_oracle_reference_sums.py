"""Pins of the reference sums: the direct O(N^2) sum (open boundary) and the
Ewald sum of Eq. refewald (periodic), with the printed formula's two defects
read as: self term -2 alpha/sqrt(pi) q_i, and q_j in the real-space term."""
import os

import numpy as np

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _madelung():
    with open(os.path.join(GOLD, "madelung.txt")) as f:
        return float([l for l in f if l.strip() and not l.startswith("#")][0])


def test_direct_two_charges():
    """Coulomb closed form: phi = q/r, grad phi = -q r/r^3."""
    pos = np.array([[0.1, 0.2, 0.3], [0.4, -0.1, 0.7]])
    q = np.array([2.0, -0.5])
    phi, g = oracle.direct(pos, q)
    d = pos[0] - pos[1]
    r = np.linalg.norm(d)
    assert abs(phi[0] - q[1] / r) < 1e-15
    assert abs(phi[1] - q[0] / r) < 1e-15
    assert np.abs(g[0] - (-q[1] * d / r ** 3)).max() < 1e-14
    assert np.abs(g[1] - (q[0] * d / r ** 3)).max() < 1e-14


def test_direct_net_force_zero():
    pos, q = synth.uniform_pm1(300, 21)
    _, g = oracle.direct(pos, q)
    F = -(q[:, None] * g)
    assert np.abs(F.sum(0)).max() < 1e-10 * np.abs(F).max()


def test_ewald_madelung():
    """NaCl lattice: phi_i = -+ M / d at every ion."""
    M = _madelung()
    for n in [2, 4]:
        pos, q = synth.rock_salt(n)
        phi, g = oracle.ewald(pos, q, (1, 1, 1), tol=1e-14)
        d = 1.0 / n
        assert np.abs(phi * d + q * M).max() < 1e-12
        assert np.abs(g).max() < 1e-10


def test_ewald_alpha_independence():
    """The Ewald sum does not depend on the splitting parameter (this fixes the sign
    of the self term: with +2 alpha/sqrt(pi) q_i it would vary as 4 alpha/sqrt(pi) q_i)."""
    pos, q = synth.uniform_pm1(256, 22)
    res = []
    for alpha in [11.0, 13.5, 16.0]:
        res.append(oracle.ewald(pos, q, (1, 1, 1), alpha, 0.5, alpha * 6.6 / np.pi))
    for phi, g in res[1:]:
        assert np.abs(phi - res[0][0]).max() < 1e-10 * np.abs(res[0][0]).max()
        assert np.abs(g - res[0][1]).max() < 1e-9 * np.abs(res[0][1]).max()


def test_ewald_neutral_net_force_and_translation():
    """Neutral periodic system: zero net force; shifting every particle by the same
    vector (with wrap) leaves every potential and force unchanged."""
    pos, q = synth.uniform_pm1(200, 23)
    phi, g = oracle.ewald(pos, q, (1, 1, 1), tol=1e-13)
    F = -(q[:, None] * g)
    assert np.abs(F.sum(0)).max() < 1e-9 * np.abs(F).max()
    pos2 = np.mod(pos + np.array([0.3141, -0.2718, 0.5772]), 1.0)
    phi2, g2 = oracle.ewald(pos2, q, (1, 1, 1), tol=1e-13)
    assert np.abs(phi2 - phi).max() < 1e-9 * np.abs(phi).max()
    assert np.abs(g2 - g).max() < 1e-8 * np.abs(g).max()


def test_ewald_rectangular_box_dipole_pair():
    """Two opposite charges in a long box: alpha-independent in a rectangular box too."""
    pos = np.array([[0.2, 0.3, 0.6], [0.9, 0.7, 1.4]])
    q = np.array([1.0, -1.0])
    box = (1.0, 1.5, 2.0)
    a1 = oracle.ewald(pos, q, box, 11.0, 0.5, 11.0 * 6.6 * 2.0 / np.pi)
    a2 = oracle.ewald(pos, q, box, 14.0, 0.5, 14.0 * 6.6 * 2.0 / np.pi)
    assert np.abs(a1[0] - a2[0]).max() < 1e-10
    assert np.abs(a1[1] - a2[1]).max() < 1e-9


def test_ewald_targets_equals_ewald():
    """The target-subset form (cell list, product phase factors) is the same sum as
    ewald(): equal on every listed target, in a cubic and a rectangular box, with
    sources outside the primary box (wrapped by the periodicity)."""
    for box in ((1.0, 1.0, 1.0), (1.0, 1.5, 2.0)):
        g = synth.rng(24)
        pos, q = synth.uniform_pm1(700, 25, length=box)
        pos[:50] += np.round(g.standard_normal((50, 3))) * np.asarray(box)
        tg = g.choice(700, size=40, replace=False)
        alpha, rcut = 14.0, 0.3
        kmax = alpha * 5.1 * max(box) / np.pi
        ref_phi, ref_g = oracle.ewald(pos, q, box, alpha, rcut, kmax, targets=tg)
        phi, gr = oracle.ewald_targets(pos, q, box, tg, alpha=alpha, rcut=rcut, kmax=kmax)
        assert np.abs(phi - ref_phi).max() < 1e-11 * np.abs(ref_phi).max()
        assert np.abs(gr - ref_g).max() < 1e-10 * np.abs(ref_g).max()


def test_ewald_targets_madelung_and_alpha():
    """Rock salt: -+ M / d at the listed ions, for two splitting parameters."""
    M = _madelung()
    pos, q = synth.rock_salt(6)
    tg = np.array([0, 1, 7, 100, 215])
    for rc in (0.25, 0.4):
        phi, gr = oracle.ewald_targets(pos, q, (1, 1, 1), tg, tol=1e-14, rcut=rc)
        assert np.abs(phi * (1.0 / 6) + q[tg] * M).max() < 1e-11
        assert np.abs(gr).max() < 1e-9
