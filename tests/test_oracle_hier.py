"""Pins of the oracle's two-level PMMM (Sec. 5, hierarchical treatment; Fig. refine):

* refine = 1 leaves the fine level empty: the result is the one-level PMMM of the
  same mesh, exactly;
* open boundary with two coarse cells per axis: every coarse pair is masked, so the
  coarse level is empty and the fine level covers every fine pair beyond the fine
  near cells: the result is the one-level PMMM of the fine mesh, to rounding;
* convergence in p against the direct sum (open) and the Ewald sum (periodic,
  neutral and charged): the error falls with p at the rate of the one-level method
  on the fine mesh and stays within a small factor of it (a dropped or mis-signed
  term of the coarse-level corrections leaves an error floor near 1e-2);
* c = 2 beats c = 1; a shift by whole coarse cells (periodic) only permutes cells.
"""
import numpy as np
import pytest

import oracle
import synth

UNIT = ((0.0, 0.0, 0.0), (1.0, 1.0, 1.0))


def _rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


@pytest.mark.parametrize("periodic", [False, True])
def test_refine1_is_one_level(periodic):
    pos, q = synth.uniform_pm1(600, 41)
    a = oracle.pmmm(pos, q, *UNIT, (8, 8, 8), 3, 1, periodic, want_ml=True)
    b = oracle.pmmm_hier(pos, q, *UNIT, (8, 8, 8), 3, 1, 1, periodic, want_ml=True)
    assert b["status"] == 0
    assert np.abs(a["phi"] - b["phi"]).max() <= 1e-14 * np.abs(a["phi"]).max()
    assert np.abs(a["grad"] - b["grad"]).max() <= 1e-14 * np.abs(a["grad"]).max()
    assert np.abs(a["L"] - b["L"]).max() <= 1e-14 * np.abs(a["L"]).max()


@pytest.mark.parametrize("refine", [2, 4])
def test_open_two_coarse_cells_is_one_level_fine(refine):
    pos, q = synth.uniform_pm1(600, 42)
    mesh = (2 * refine,) * 3
    a = oracle.pmmm(pos, q, *UNIT, mesh, 4, 1, False, want_ml=True)
    b = oracle.pmmm_hier(pos, q, *UNIT, mesh, 4, refine, 1, False, want_ml=True)
    assert np.abs(a["phi"] - b["phi"]).max() < 1e-12 * np.abs(a["phi"]).max()
    assert np.abs(a["grad"] - b["grad"]).max() < 1e-12 * np.abs(a["grad"]).max()
    assert np.abs(a["L"] - b["L"]).max() < 1e-12 * np.abs(a["L"]).max()


def _sample_cells(pos, mesh, n, seed, periodic=False):
    st, cell, perm, cs, w = oracle.bin_particles(pos, *UNIT, mesh, periodic)
    occ = np.nonzero(np.diff(cs))[0]
    tc = synth.rng(seed).choice(occ, min(n, occ.size), replace=False)
    return tc, np.isin(cell, tc)


def test_open_convergence_against_direct():
    pos, q = synth.paper_sec4(2048, 32)
    mesh = (16, 16, 16)
    tc, sel = _sample_cells(pos, mesh, 120, 43)
    ph, g = oracle.direct(pos, q, targets=np.nonzero(sel)[0])
    e_h, e_u = [], []
    for p in (1, 3, 5, 7):
        rh = oracle.pmmm_hier(pos, q, *UNIT, mesh, p, 4, 1, False, target_cells=tc)
        ru = oracle.pmmm(pos, q, *UNIT, mesh, p, 1, False, target_cells=tc)
        e_h.append(_rel(rh["grad"][sel], g))
        e_u.append(_rel(ru["grad"][sel], g))
    assert all(b < 0.25 * a for a, b in zip(e_h, e_h[1:])), e_h
    assert all(h < 1.3 * u for h, u in zip(e_h, e_u)), (e_h, e_u)
    assert e_h[-1] < 3e-4


@pytest.mark.parametrize("charged,refine", [(False, 2), (True, 4)])
def test_periodic_convergence_against_ewald(charged, refine):
    pos, q = synth.paper_sec4(1024, 35)
    if charged:
        q = q + 0.5 / 1024.0
    ph, g = oracle.ewald(pos, q, (1, 1, 1), tol=1e-13)
    eg, ep = [], []
    for p in (2, 4, 6, 8):
        r = oracle.pmmm_hier(pos, q, *UNIT, (16, 16, 16), p, refine, 1, True, nmax=6)
        eg.append(_rel(r["grad"], g))
        ep.append(_rel(r["phi"], ph))
    assert all(b < 0.3 * a for a, b in zip(eg, eg[1:])), (refine, eg)
    assert all(b < 0.3 * a for a, b in zip(ep, ep[1:])), (refine, ep)
    assert eg[-1] < 1.5e-4 and ep[-1] < 5e-5, (refine, eg, ep)


def test_cutoff2_beats_cutoff1():
    pos, q = synth.paper_sec4(2048, 44)
    mesh = (16, 16, 16)
    tc, sel = _sample_cells(pos, mesh, 60, 45, periodic=True)
    ph, g = oracle.ewald(pos, q, (1, 1, 1), tol=1e-13, targets=np.nonzero(sel)[0])
    e = {}
    for c in (1, 2):
        r = oracle.pmmm_hier(pos, q, *UNIT, mesh, 5, 2, c, True, nmax=6, target_cells=tc)
        e[c] = (_rel(r["grad"][sel], g), _rel(r["phi"][sel], ph))
    assert e[2][0] < 0.5 * e[1][0] and e[2][1] < 0.5 * e[1][1], e


def test_periodic_shift_by_coarse_cells():
    pos, q = synth.uniform_pm1(1024, 46)
    r = oracle.pmmm_hier(pos, q, *UNIT, (16, 16, 16), 3, 4, 1, True, nmax=5)
    pos2 = np.mod(pos + np.array([1, 3, 2]) / 4.0, 1.0)
    r2 = oracle.pmmm_hier(pos2, q, *UNIT, (16, 16, 16), 3, 4, 1, True, nmax=5)
    assert np.abs(r2["phi"] - r["phi"]).max() < 1e-9 * np.abs(r["phi"]).max()
    assert np.abs(r2["grad"] - r["grad"]).max() < 1e-9 * np.abs(r["grad"]).max()
