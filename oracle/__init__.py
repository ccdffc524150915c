"""FP64 CPU oracle for the particle mesh multipole method (arXiv:1409.5981).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The GPU library and
its Python binding never import, link or call it, and share no code with it.

The arithmetic lives in ``pmmm_oracle.c`` (plain C loops, double precision,
written from the paper's definitions; see the header of that file for the
equation each routine follows).  This module compiles it with gcc on first use
and wraps it with ctypes and numpy.

Parity pins: every routine here is checked in ``tests/test_oracle_*.py`` against
something other than itself (the paper's table of low-order harmonics, scipy /
sympy Legendre functions, addition theorems, closed forms, the Madelung
constant, alpha-independence, brute-force lattice sums, a numpy FFT convolution
at p = 0).  Nothing is marked "parity unpinned".

Complex harmonic arrays use the full index ``l*l + l + m`` (m in [-l, l]).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pmmm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

OK, ERR_OUT_OF_BOX, ERR_NONFINITE = 0, -3, -4


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            d, i32, i64, vp = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
            sig = {
                "orc_version": (i32, []),
                "orc_max_threads": (i32, []),
                "orc_set_threads": (None, [i32]),
                "orc_legendre": (None, [i32, d, d, vp]),
                "orc_solid_R": (None, [i32, vp, vp]),
                "orc_solid_S": (None, [i32, vp, vp]),
                "orc_gammaQ_half": (d, [i32, d]),
                "orc_gammaP_half": (d, [i32, d]),
                "orc_p2m": (None, [i32, i64, vp, vp, vp, vp]),
                "orc_m2m": (None, [i32, vp, vp, vp]),
                "orc_m2p": (d, [i32, vp, vp]),
                "orc_m2l": (None, [i32, vp, vp, vp]),
                "orc_m2l_green": (None, [i32, vp, vp, vp]),
                "orc_l2l": (None, [i32, i32, vp, vp, vp]),
                "orc_l2p": (None, [i32, vp, vp, vp, vp]),
                "orc_l2p_phi": (d, [i32, vp, vp]),
                "orc_direct": (None, [i64, vp, vp, i64, vp, vp, vp]),
                "orc_ewald": (None, [i64, vp, vp, vp, d, d, d, i64, vp, vp, vp]),
                "orc_ewald_targets": (i32, [i64, vp, vp, vp, d, d, d, i64, vp, vp, vp]),
                "orc_bin": (i32, [i64, vp, vp, vp, vp, i32, vp, vp, vp, vp]),
                "orc_green_open": (None, [i32, i32, vp, vp, vp]),
                "orc_green_periodic": (None, [i32, i32, vp, vp, d, i32, vp, vp]),
                "orc_pmmm": (i32, [vp, i64, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp]),
                "orc_pmmm_hier": (i32, [vp, i32, i64, vp, vp, i64, vp, vp, vp, vp, vp, vp]),
                "orc_green_table_size": (i64, [vp]),
                "orc_green_table": (None, [vp, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def threads() -> int:
    """Number of OpenMP threads the oracle uses."""
    return int(_L().orc_max_threads())


def set_threads(n: int) -> None:
    _L().orc_set_threads(int(n))


def nterms(p: int) -> int:
    return (p + 1) * (p + 1)


def hidx(l: int, m: int) -> int:
    return l * l + l + m


# --------------------------------------------------------------------------- harmonics
def legendre(lmax: int, x: float, s: float | None = None) -> np.ndarray:
    """P_l^m(x) for 0<=m<=l<=lmax at index hidx(l, m) (App. A.1 definition)."""
    if s is None:
        s = math.sqrt(max(0.0, 1.0 - x * x))
    out = np.zeros(nterms(lmax))
    _L().orc_legendre(lmax, float(x), float(s), _p(out))
    return out


def solid_R(p: int, r) -> np.ndarray:
    r = _f64(r, (3,))
    out = np.zeros(nterms(p), dtype=np.complex128)
    _L().orc_solid_R(p, _p(r), _p(out))
    return out


def solid_S(p: int, r) -> np.ndarray:
    r = _f64(r, (3,))
    out = np.zeros(nterms(p), dtype=np.complex128)
    _L().orc_solid_S(p, _p(r), _p(out))
    return out


def gammaQ_half(l: int, x: float) -> float:
    """Gamma(l+1/2, x) / Gamma(l+1/2)."""
    return float(_L().orc_gammaQ_half(l, float(x)))


def gammaP_half(l: int, x: float) -> float:
    """gamma(l+1/2, x) / Gamma(l+1/2)."""
    return float(_L().orc_gammaP_half(l, float(x)))


# --------------------------------------------------------------------------- translations
def p2m(p: int, pos, q, center) -> np.ndarray:
    pos = _f64(pos).reshape(-1, 3)
    q = _f64(q).reshape(-1)
    c = _f64(center, (3,))
    M = np.zeros(nterms(p), dtype=np.complex128)
    _L().orc_p2m(p, pos.shape[0], _p(pos), _p(q), _p(c), _p(M))
    return M


def m2m(p: int, M, shift) -> np.ndarray:
    M = np.ascontiguousarray(M, dtype=np.complex128)
    s = _f64(shift, (3,))
    out = np.zeros(nterms(p), dtype=np.complex128)
    _L().orc_m2m(p, _p(M), _p(s), _p(out))
    return out


def m2p(p: int, M, r) -> float:
    M = np.ascontiguousarray(M, dtype=np.complex128)
    r = _f64(r, (3,))
    return float(_L().orc_m2p(p, _p(M), _p(r)))


def m2l(p: int, M, d, L=None) -> np.ndarray:
    """L += M2L(M) for r_L - r_M = d."""
    M = np.ascontiguousarray(M, dtype=np.complex128)
    d = _f64(d, (3,))
    L = np.zeros(nterms(p), dtype=np.complex128) if L is None else np.ascontiguousarray(L, dtype=np.complex128)
    _L().orc_m2l(p, _p(M), _p(d), _p(L))
    return L


def m2l_green(p: int, M, G, L=None) -> np.ndarray:
    M = np.ascontiguousarray(M, dtype=np.complex128)
    G = np.ascontiguousarray(G, dtype=np.complex128)
    L = np.zeros(nterms(p), dtype=np.complex128) if L is None else np.ascontiguousarray(L, dtype=np.complex128)
    _L().orc_m2l_green(p, _p(M), _p(G), _p(L))
    return L


def l2l(p: int, pout: int, L, shift) -> np.ndarray:
    L = np.ascontiguousarray(L, dtype=np.complex128)
    s = _f64(shift, (3,))
    out = np.zeros(nterms(pout), dtype=np.complex128)
    _L().orc_l2l(p, pout, _p(L), _p(s), _p(out))
    return out


def l2p(p: int, L, r):
    """(phi, grad) at r - r_L = r: Eq. L2P and the order-one L2L gradient (Eq. phigrad)."""
    L = np.ascontiguousarray(L, dtype=np.complex128)
    r = _f64(r, (3,))
    phi = np.zeros(1)
    g = np.zeros(3)
    _L().orc_l2p(p, _p(L), _p(r), _p(phi), _p(g))
    return float(phi[0]), g


def l2p_phi(p: int, L, r) -> float:
    L = np.ascontiguousarray(L, dtype=np.complex128)
    r = _f64(r, (3,))
    return float(_L().orc_l2p_phi(p, _p(L), _p(r)))


# --------------------------------------------------------------------------- reference sums
def direct(pos, q, targets=None):
    """Open-boundary O(N^2) sum: (phi, grad) for the targets (all if None)."""
    pos = _f64(pos).reshape(-1, 3)
    q = _f64(q).reshape(-1)
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = pos.shape[0] if t is None else t.shape[0]
    phi = np.zeros(nt)
    g = np.zeros((nt, 3))
    _L().orc_direct(pos.shape[0], _p(pos), _p(q), nt, _p(t), _p(phi), _p(g))
    return phi, g


def ewald_params(box, tol: float = 1e-10, n_targets: int | None = None, n_sources: int | None = None):
    """A (alpha, rcut, kmax) triple with real-space cutoff at most half the
    smallest box side and both truncations below ~tol (erfc and Gaussian)."""
    b = float(min(box))
    s = math.sqrt(-math.log(tol)) + 0.5
    rcut = 0.5 * b
    alpha = s / rcut
    kmax = s * alpha * max(box) / math.pi
    return alpha, rcut, kmax


def ewald(pos, q, box, alpha=None, rcut=None, kmax=None, targets=None, tol: float = 1e-10):
    """Periodic Ewald reference (Eq. refewald): (phi, grad) for the targets."""
    pos = _f64(pos).reshape(-1, 3)
    q = _f64(q).reshape(-1)
    box = _f64(box, (3,))
    if alpha is None:
        alpha, rcut, kmax = ewald_params(box, tol)
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = pos.shape[0] if t is None else t.shape[0]
    phi = np.zeros(nt)
    g = np.zeros((nt, 3))
    _L().orc_ewald(pos.shape[0], _p(pos), _p(q), _p(box), float(alpha), float(rcut), float(kmax), nt, _p(t),
                   _p(phi), _p(g))
    return phi, g


def ewald_targets(pos, q, box, targets, tol: float = 1e-9, rcut: float | None = None, alpha=None, kmax=None):
    """The Ewald sum of Eq. refewald for a few targets among many sources: (phi, grad)
    of the listed targets.  The same sum as ewald(); the real-space part visits only
    cells of side >= rcut around each target and the structure factors use products
    of per-axis phase factors, which keeps N = 2^20 sources affordable.  By default
    rcut = 0.3 b_min, alpha and kmax from tol as in ewald_params."""
    pos = _f64(pos).reshape(-1, 3)
    q = _f64(q).reshape(-1)
    box = _f64(box, (3,))
    t = np.ascontiguousarray(targets, dtype=np.int64)
    if alpha is None:
        s = math.sqrt(-math.log(tol)) + 0.5
        rcut = 0.3 * float(min(box)) if rcut is None else float(rcut)
        alpha = s / rcut
        kmax = s * alpha * float(max(box)) / math.pi
    phi = np.zeros(t.shape[0])
    g = np.zeros((t.shape[0], 3))
    st = _L().orc_ewald_targets(pos.shape[0], _p(pos), _p(q), _p(box), float(alpha), float(rcut), float(kmax),
                                t.shape[0], _p(t), _p(phi), _p(g))
    if st != 0:
        raise ValueError("ewald_targets needs rcut <= 3b/7 on every axis")
    return phi, g


# --------------------------------------------------------------------------- binning
def bin_particles(pos, lo, length, mesh, periodic: bool):
    """(status, cell id per particle, stable permutation, cell_start[K+1], binned coordinates)."""
    pos = _f64(pos).reshape(-1, 3)
    lo = _f64(lo, (3,))
    ln = _f64(length, (3,))
    mesh = np.ascontiguousarray(mesh, dtype=np.int32).reshape(3)
    n = pos.shape[0]
    K = int(mesh[0]) * int(mesh[1]) * int(mesh[2])
    cell = np.zeros(n, dtype=np.int32)
    perm = np.zeros(n, dtype=np.int64)
    cs = np.zeros(K + 1, dtype=np.int64)
    w = np.zeros((n, 3))
    st = _L().orc_bin(n, _p(pos), _p(lo), _p(ln), _p(mesh), int(bool(periodic)), _p(cell), _p(perm), _p(cs), _p(w))
    return int(st), cell, perm, cs, w


# --------------------------------------------------------------------------- Green functions
def green_open(p: int, c: int, h, d) -> np.ndarray:
    h = _f64(h, (3,))
    d = np.ascontiguousarray(d, dtype=np.int32).reshape(3)
    G = np.zeros(nterms(2 * p), dtype=np.complex128)
    _L().orc_green_open(p, c, _p(h), _p(d), _p(G))
    return G


def green_periodic(p: int, c: int, mesh, box, alpha: float, nmax: int, d) -> np.ndarray:
    mesh = np.ascontiguousarray(mesh, dtype=np.int32).reshape(3)
    box = _f64(box, (3,))
    d = np.ascontiguousarray(d, dtype=np.int32).reshape(3)
    G = np.zeros(nterms(2 * p), dtype=np.complex128)
    _L().orc_green_periodic(p, c, _p(mesh), _p(box), float(alpha), int(nmax), _p(d), _p(G))
    return G


# --------------------------------------------------------------------------- PMMM
class _Cfg(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("len", ctypes.c_double * 3), ("mesh", ctypes.c_int * 3),
                ("p", ctypes.c_int), ("c", ctypes.c_int), ("periodic", ctypes.c_int),
                ("alpha", ctypes.c_double), ("nmax", ctypes.c_int)]


def default_alpha(box) -> float:
    """alpha * b = 1.5 on the smallest box side (App. B.1 example for a unit box)."""
    return 1.5 / float(min(box))


def _cfg(lo, length, mesh, p, c, periodic, alpha, nmax) -> _Cfg:
    cfg = _Cfg()
    for a in range(3):
        cfg.lo[a] = float(lo[a])
        cfg.len[a] = float(length[a])
        cfg.mesh[a] = int(mesh[a])
    cfg.p, cfg.c, cfg.periodic = int(p), int(c), int(bool(periodic))
    cfg.alpha = float(default_alpha(length) if alpha is None else alpha)
    cfg.nmax = int(nmax)
    return cfg


def green_table(lo, length, mesh, p: int, c: int = 1, periodic: bool = False, alpha: float | None = None,
                nmax: int = 5) -> np.ndarray:
    """Green function of every distinct cell displacement (the set-up step of Sec. 2.1),
    to pass to pmmm(..., green=...) for repeated evaluations with the same geometry."""
    cfg = _cfg(lo, length, mesh, p, c, periodic, alpha, nmax)
    ng = _L().orc_green_table_size(ctypes.byref(cfg))
    out = np.zeros((ng, nterms(2 * p)), dtype=np.complex128)
    _L().orc_green_table(ctypes.byref(cfg), _p(out))
    return out


def pmmm(pos, q, lo, length, mesh, p: int, c: int = 1, periodic: bool = False, alpha: float | None = None,
         nmax: int = 5, target_cells=None, want_ml: bool = False, green: np.ndarray | None = None):
    """PMMM by its definition: all-cell-pair convolution, corrections, L2P, near field.

    Returns dict(status, phi, grad, [M, L, corr]).  phi/grad (Coulomb sign, grad = grad Phi)
    are filled for the particles of the target cells (all cells if None), NaN elsewhere.
    M: (K, (p+1)^2) complex multipoles; L: (K, (p+1)^2) complex locals after the
    convolution (before corrections) for the target cells, zeros elsewhere.
    green: optional table from green_table() with the same geometry.
    """
    pos = _f64(pos).reshape(-1, 3)
    q = _f64(q).reshape(-1)
    cfg = _cfg(lo, length, mesh, p, c, periodic, alpha, nmax)
    n = pos.shape[0]
    K = int(mesh[0]) * int(mesh[1]) * int(mesh[2])
    tc = None if target_cells is None else np.ascontiguousarray(target_cells, dtype=np.int64)
    ntc = -1 if tc is None else tc.shape[0]
    phi = np.full(n, np.nan)
    g = np.full((n, 3), np.nan)
    M = np.zeros((K, nterms(p)), dtype=np.complex128) if want_ml else None
    Lo = np.zeros((K, nterms(p)), dtype=np.complex128) if want_ml else None
    corr = np.zeros(8)
    if green is not None:
        green = np.ascontiguousarray(green, dtype=np.complex128)
        if green.shape != (_L().orc_green_table_size(ctypes.byref(cfg)), nterms(2 * p)):
            raise ValueError("green table does not match the geometry")
    st = _L().orc_pmmm(ctypes.byref(cfg), n, _p(pos), _p(q), ntc, _p(tc), _p(phi), _p(g), _p(M), _p(Lo), _p(corr),
                       _p(green))
    out = {"status": int(st), "phi": phi, "grad": g, "corr": corr, "alpha": cfg.alpha}
    if want_ml:
        out["M"] = M
        out["L"] = Lo
    return out


def pmmm_hier(pos, q, lo, length, mesh, p: int, refine: int, c: int = 1, periodic: bool = False,
              alpha: float | None = None, nmax: int = 5, target_cells=None, want_ml: bool = False,
              green_coarse: np.ndarray | None = None):
    """Two-level PMMM (Sec. 5, hierarchical treatment) by its definition: PMMM on the
    coarse mesh (mesh / refine cells per axis, the coarse (2c+1)^3 block masked),
    free-space M2L between the fine cells of the masked coarse block (fine (2c+1)^3
    block masked), near field over the fine (2c+1)^3 cells.

    `mesh` is the fine mesh.  Returns dict(status, phi, grad, [M, L]) like pmmm():
    M the fine multipoles, L per target fine cell the total local expansion before the
    periodic corrections, L2L(coarse local) + the fine-level sum.
    green_coarse: optional green_table() of the coarse geometry."""
    pos = _f64(pos).reshape(-1, 3)
    q = _f64(q).reshape(-1)
    cfg = _cfg(lo, length, mesh, p, c, periodic, alpha, nmax)
    n = pos.shape[0]
    K = int(mesh[0]) * int(mesh[1]) * int(mesh[2])
    tc = None if target_cells is None else np.ascontiguousarray(target_cells, dtype=np.int64)
    ntc = -1 if tc is None else tc.shape[0]
    phi = np.full(n, np.nan)
    g = np.full((n, 3), np.nan)
    M = np.zeros((K, nterms(p)), dtype=np.complex128) if want_ml else None
    Lo = np.zeros((K, nterms(p)), dtype=np.complex128) if want_ml else None
    if green_coarse is not None:
        green_coarse = np.ascontiguousarray(green_coarse, dtype=np.complex128)
    st = _L().orc_pmmm_hier(ctypes.byref(cfg), int(refine), n, _p(pos), _p(q), ntc, _p(tc), _p(phi), _p(g), _p(M),
                            _p(Lo), _p(green_coarse))
    out = {"status": int(st), "phi": phi, "grad": g, "alpha": cfg.alpha}
    if want_ml:
        out["M"] = M
        out["L"] = Lo
    return out


def error_estimate(c: int, p: int) -> float:
    """Worst-case relative error of Eq. errest: ((sqrt3/2) / ((c+1) - sqrt3/2))^(p+1)."""
    a = math.sqrt(3.0) / 2.0
    return (a / ((c + 1) - a)) ** (p + 1)


def to_real_storage(X: np.ndarray) -> np.ndarray:
    """Complex full-index harmonics -> the real storage of App. A.7:
    X_{l(l+1)+m} = Re X_l^{|m|} (m >= 0), Im X_l^{|m|} (m < 0).  Works on the last axis."""
    X = np.asarray(X)
    nt = X.shape[-1]
    p = int(round(math.sqrt(nt))) - 1
    out = np.zeros(X.shape, dtype=np.float64)
    for l in range(p + 1):
        for m in range(-l, l + 1):
            src = X[..., hidx(l, abs(m))]
            out[..., hidx(l, m)] = src.real if m >= 0 else src.imag
    return out
