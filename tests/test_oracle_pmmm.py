"""Pins of the oracle's whole PMMM (Sec. 2.1 cell-pair definition, Sec. 2.2,
App. B.3) to the physical references and to special cases:

* open boundary, one particle at each occupied cell centre: PMMM == direct sum
  exactly (only l = 0 moments, and the local expansion is evaluated at its centre);
* periodic, particles at cell centres: PMMM == Ewald (App. B.3 remark), which on
  the rock-salt lattice gives the Madelung constant;
* error against direct / Ewald falls with p, no slower than Eq. errest, and c = 2
  beats c = 1 (Sec. 3.2, Sec. 4);
* p = 0 is the PM method in NGP mode (Sec. 2.2): the far field equals a numpy FFT
  convolution of the cell charge grid with the masked 1/r kernel;
* invariances: alpha, shifts by whole cells, zero net force (neutral periodic).
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
UNIT = ((0.0, 0.0, 0.0), (1.0, 1.0, 1.0))


def _rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def test_open_cell_centres_equal_direct():
    pos, q = synth.cell_centres((6, 6, 6), (0, 0, 0), (1, 1, 1), 31, fill=0.5)
    ph, g = oracle.direct(pos, q)
    for p in (0, 1, 3, 5):
        r = oracle.pmmm(pos, q, *UNIT, (6, 6, 6), p, 1, False)
        assert np.abs(r["phi"] - ph).max() < 1e-12 * np.abs(ph).max()
        if p >= 1:
            assert np.abs(r["grad"] - g).max() < 1e-12 * np.abs(g).max()


def test_open_convergence_in_p_and_cutoff():
    pos, q = synth.paper_sec4(2048, 32)
    ph, g = oracle.direct(pos, q)
    errs = {}
    for c in (1, 2):
        for p in (1, 3, 5, 7):
            r = oracle.pmmm(pos, q, *UNIT, (8, 8, 8), p, c, False)
            errs[c, p] = (_rel(r["phi"], ph), _rel(r["grad"], g))
    for c in (1, 2):
        e = [errs[c, p][1] for p in (1, 3, 5, 7)]
        assert all(b < a for a, b in zip(e, e[1:])), e
        # Eq. errest is a worst-case bound per order; the observed rate is at least as fast
        rate = (e[-1] / e[0]) ** (1.0 / 6.0)
        assert rate < oracle.error_estimate(c, 1) / oracle.error_estimate(c, 0) + 0.05, (c, rate)
    for p in (3, 5, 7):
        assert errs[2, p][1] < errs[1, p][1]
        assert errs[2, p][0] < errs[1, p][0]


def test_periodic_rock_salt_madelung():
    with open(os.path.join(GOLD, "madelung.txt")) as f:
        M = float([l for l in f if l.strip() and not l.startswith("#")][0])
    pos, q = synth.rock_salt(8)
    for p in (1, 4):
        r = oracle.pmmm(pos, q, *UNIT, (8, 8, 8), p, 1, True, nmax=6)
        assert np.abs(r["phi"] / 8.0 + q * M).max() < 1e-11
        assert np.abs(r["grad"]).max() < 1e-10


@pytest.mark.parametrize("charged", [False, True])
def test_periodic_cell_centres_equal_ewald(charged):
    pos, q = synth.cell_centres((8, 8, 8), (0, 0, 0), (1, 1, 1), 33, fill=0.3)
    if not charged:
        q -= q.mean()
    ph, g = oracle.ewald(pos, q, (1, 1, 1), tol=1e-14)
    r = oracle.pmmm(pos, q, *UNIT, (8, 8, 8), 3, 1, True, nmax=6)
    assert np.abs(r["phi"] - ph).max() < 1e-10 * np.abs(ph).max()
    assert np.abs(r["grad"] - g).max() < 1e-10 * np.abs(g).max()


def test_periodic_convergence_and_alpha_independence():
    pos, q = synth.uniform_pm1(1024, 34)
    ph, g = oracle.ewald(pos, q, (1, 1, 1), tol=1e-13)
    e = []
    for p in (1, 3, 5):
        r = oracle.pmmm(pos, q, *UNIT, (8, 8, 8), p, 1, True, nmax=6)
        e.append(_rel(r["grad"], g))
    assert all(b < a for a, b in zip(e, e[1:]))
    assert e[-1] < 1e-3
    # alpha only moves work between the two lattice sums
    r1 = oracle.pmmm(pos, q, *UNIT, (8, 8, 8), 3, 1, True, alpha=1.5, nmax=7)
    r2 = oracle.pmmm(pos, q, *UNIT, (8, 8, 8), 3, 1, True, alpha=2.4, nmax=7)
    assert np.abs(r1["phi"] - r2["phi"]).max() < 1e-10 * np.abs(r1["phi"]).max()
    assert np.abs(r1["grad"] - r2["grad"]).max() < 1e-10 * np.abs(r1["grad"]).max()


def test_periodic_charged_system():
    pos, q = synth.paper_sec4(1024, 35)
    q = q + 0.5 / 1024.0
    ph, g = oracle.ewald(pos, q, (1, 1, 1), tol=1e-13)
    e = []
    for p in (2, 4, 6):
        r = oracle.pmmm(pos, q, *UNIT, (8, 8, 8), p, 1, True, nmax=6)
        e.append((_rel(r["phi"], ph), _rel(r["grad"], g)))
    assert all(b[1] < a[1] for a, b in zip(e, e[1:]))
    assert e[-1][1] < 2e-3 and e[-1][0] < 1e-3


def test_periodic_net_force_small_and_shift_invariance():
    pos, q = synth.uniform_pm1(1024, 36)
    fn = []
    for p in (2, 5):
        r = oracle.pmmm(pos, q, *UNIT, (8, 8, 8), p, 1, True, nmax=5)
        F = -(q[:, None] * r["grad"])
        # truncation errors of the N forces add like a random walk: compare the net
        # force with the root of the summed squared forces
        fn.append(np.abs(F.sum(0)).max() / np.sqrt((F ** 2).sum()))
    assert fn[1] < fn[0] and fn[1] < 2e-3
    # whole-cell shift with wrap: same cells, permuted -> identical results
    r = oracle.pmmm(pos, q, *UNIT, (8, 8, 8), 3, 1, True, nmax=5)
    pos2 = np.mod(pos + np.array([3, 1, 6]) / 8.0, 1.0)
    r2 = oracle.pmmm(pos2, q, *UNIT, (8, 8, 8), 3, 1, True, nmax=5)
    assert np.abs(r2["phi"] - r["phi"]).max() < 1e-9 * np.abs(r["phi"]).max()
    assert np.abs(r2["grad"] - r["grad"]).max() < 1e-9 * np.abs(r["grad"]).max()


def test_p0_is_pm_ngp_convolution():
    """Sec. 2.2: at p = 0 the cell convolution is the scalar NGP PM convolution.
    Checked against numpy's FFT on a 2n zero-padded grid with the masked 1/r kernel."""
    n, c = 8, 1
    pos, q = synth.uniform_pm1(600, 37)
    r = oracle.pmmm(pos, q, *UNIT, (n, n, n), 0, c, False, want_ml=True)
    st, cell, perm, cs, _ = oracle.bin_particles(pos, (0, 0, 0), (1, 1, 1), (n, n, n), False)
    rho = np.bincount(cell, weights=q, minlength=n ** 3).reshape(n, n, n)  # [z][y][x]
    L2 = 2 * n
    ker = np.zeros((L2, L2, L2))
    h = 1.0 / n
    for dz in range(-(n - 1), n):
        for dy in range(-(n - 1), n):
            for dx in range(-(n - 1), n):
                if max(abs(dx), abs(dy), abs(dz)) <= c:
                    continue
                ker[dz % L2, dy % L2, dx % L2] = 1.0 / (h * np.sqrt(dx * dx + dy * dy + dz * dz))
    pad = np.zeros((L2, L2, L2))
    pad[:n, :n, :n] = rho
    conv = np.real(np.fft.ifftn(np.fft.fftn(pad) * np.fft.fftn(ker)))[:n, :n, :n].reshape(-1)
    L00 = r["L"][:, 0].real
    assert np.abs(L00 - conv).max() < 1e-11 * np.abs(conv).max()


def test_binning_faces_wrap_and_errors():
    lo, ln, mesh = (0.0, -1.0, 2.0), (1.0, 2.0, 4.0), (4, 8, 2)
    # points exactly on cell faces (dyadic, exactly representable) land in the upper cell
    pts = np.array([[0.25, -1.0, 2.0], [0.5, -0.75, 4.0], [0.75, 0.0, 5.999999999999999], [0.0, 0.99999999999999, 2.0]])
    st, cell, perm, cs, _ = oracle.bin_particles(pts, lo, ln, mesh, False)
    assert st == 0
    assert list(cell) == [1 + 4 * (0 + 8 * 0), 2 + 4 * (1 + 8 * 1), 3 + 4 * (4 + 8 * 1), 0 + 4 * (7 + 8 * 0)]
    # stable order within a cell and the CSR offsets
    pts2 = np.array([[0.1, -0.9, 2.1], [0.9, 0.9, 5.9], [0.12, -0.95, 2.2], [0.11, -0.99, 2.3]])
    st, cell, perm, cs, _ = oracle.bin_particles(pts2, lo, ln, mesh, False)
    assert list(perm) == [0, 2, 3, 1]
    assert cs[0] == 0 and cs[1] == 3 and cs[-1] == 4
    # open boundary: a point outside the box is an error; NaN is an error
    st, *_ = oracle.bin_particles(np.array([[1.0, 0.0, 3.0]]), lo, ln, mesh, False)
    assert st == oracle.ERR_OUT_OF_BOX
    st, *_ = oracle.bin_particles(np.array([[np.nan, 0.0, 3.0]]), lo, ln, mesh, False)
    assert st == oracle.ERR_NONFINITE
    # periodic: wrapped into the box
    st, cell, perm, cs, w = oracle.bin_particles(np.array([[1.25, -1.5, 7.0], [-0.25, 3.0, 1.0]]), lo, ln, mesh, True)
    assert st == 0
    assert np.allclose(w, [[0.25, 0.5, 3.0], [0.75, -1.0, 5.0]])
    assert list(cell) == [1 + 4 * (6 + 8 * 0), 3 + 4 * (0 + 8 * 1)]


def test_fixed_error_order_per_cutoff():
    """The error axis of the headline metric: relative RMS force error against Ewald
    (Eq. refewald) of the bench's distribution (uniform, 32 particles per cell, +-1
    charges, periodic) for p = 2..8 (c = 1) and 2..6 (c = 2), on all particles of 32
    seeded cells of an 8^3 mesh.  It falls by a constant ratio per order, faster than Eq. errest's
    worst-case ratio, c = 2 below c = 1; the lowest order at a relative RMS force error
    <= 1e-4 is p = 7 for c = 1 (the bench's order) and p = 4 for c = 2."""
    n, m = 16384, 8
    pos, q = synth.uniform_pm1(n, synth.seed(2, 77))
    cells = synth.rng(synth.seed(2, 78)).choice(m ** 3, size=32, replace=False)
    _, cell, *_ = oracle.bin_particles(pos, *UNIT, (m,) * 3, True)
    tg = np.nonzero(np.isin(cell, cells))[0]
    _, g_e = oracle.ewald(pos, q, (1, 1, 1), targets=tg)
    lowest = {}
    for c, orders in ((1, range(2, 9)), (2, range(2, 7))):
        e = []
        for p in orders:
            r = oracle.pmmm(pos, q, *UNIT, (m,) * 3, p, c, True, target_cells=cells)
            g = r["grad"][tg]
            e.append(float(np.sqrt((q[tg, None] ** 2 * (g - g_e) ** 2).sum() / (q[tg, None] ** 2 * g_e ** 2).sum())))
        print(f"c = {c}: force error vs Ewald " + ", ".join(f"p={p} {x:.2e}" for p, x in zip(orders, e)))
        assert all(b < a for a, b in zip(e, e[1:])), e
        rate = (e[-1] / e[0]) ** (1.0 / (len(e) - 1))
        assert rate < oracle.error_estimate(c, 1) / oracle.error_estimate(c, 0), (c, rate)
        lowest[c] = next(p for p, x in zip(orders, e) if x <= 1e-4)
        if c == 2:  # same orders: c = 2 below c = 1
            assert all(x2 < x1 for x2, x1 in zip(e, e1)), (e, e1)
        e1 = e
    assert lowest == {1: 7, 2: 4}, lowest
