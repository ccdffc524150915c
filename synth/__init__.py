"""Seeded synthetic inputs shared by the tests, the oracle checks and bench.py.

This module holds no arithmetic of the method: it only draws particle
positions and charges (numpy PCG64 generators), with the shapes and
distributions of the paper's test (Sec. 4) and of the benchmark workloads.
No public dataset is involved anywhere.

Seed convention: ``seed(config, rep) = 1409598 + 1000 * config + rep``.
"""
from __future__ import annotations

import numpy as np


def seed(config: int, rep: int = 0) -> int:
    return 1409598 + 1000 * int(config) + int(rep)


def rng(s: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(s)))


def uniform_pm1(n: int, s: int, lo=(0.0, 0.0, 0.0), length=(1.0, 1.0, 1.0)):
    """n points uniform in the box, charges +1/-1 with exactly n//2 of each
    (one charge 0 when n is odd), shuffled: a neutral system."""
    g = rng(s)
    lo = np.asarray(lo, dtype=np.float64)
    length = np.asarray(length, dtype=np.float64)
    pos = lo + g.random((n, 3)) * length
    q = np.zeros(n)
    q[: n // 2] = 1.0
    q[n // 2: 2 * (n // 2)] = -1.0
    g.shuffle(q)
    return pos, q


def paper_sec4(n: int, s: int):
    """Sec. 4 test condition: uniform in the unit box, charges uniform in [0, 1/n)
    then shifted by their mean so that the total charge is zero."""
    g = rng(s)
    pos = g.random((n, 3))
    q = g.random(n) / n
    q -= q.mean()
    return pos, q


def plummer(n: int, s: int, a: float = 0.1, rmax_over_a: float = 10.0):
    """Plummer sphere centred at the origin: r = a / sqrt(X^(-2/3) - 1), radii above
    rmax rejected, isotropic directions, equal masses 1/n.  Box [-1, 1]^3 holds it."""
    g = rng(s)
    out = np.empty((0, 3))
    rmax = a * rmax_over_a
    while out.shape[0] < n:
        m = 2 * (n - out.shape[0]) + 16
        X = g.random(m)
        X = X[(X > 0.0)]
        r = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
        r = r[r <= rmax]
        k = r.shape[0]
        ct = 2.0 * g.random(k) - 1.0
        ph = 2.0 * np.pi * g.random(k)
        st = np.sqrt(1.0 - ct * ct)
        pts = np.stack([r * st * np.cos(ph), r * st * np.sin(ph), r * ct], axis=1)
        out = np.concatenate([out, pts], axis=0)
    pos = out[:n]
    q = np.full(n, 1.0 / n)
    return pos, q


def batched_sizes(nsys: int, s: int, lo_exp: float = 14.0, hi_exp: float = 18.0):
    """System sizes N = 2 * round(2^(lo + (hi-lo) u) / 2), u ~ U[0, 1): log-uniform, even."""
    g = rng(s)
    u = g.random(nsys)
    return (2 * np.round(2.0 ** (lo_exp + (hi_exp - lo_exp) * u) / 2.0)).astype(np.int64)


def batched_uniform_pm1(sizes, config: int, rep: int = 0, lo=(0.0, 0.0, 0.0), length=(1.0, 1.0, 1.0)):
    """Independent neutral uniform +-1 systems of the given sizes, system s drawn from
    seed(config, 100 * rep + s); returns the concatenated (pos, q) and the offsets."""
    pos, q = [], []
    for s, n in enumerate(sizes):
        a, b = uniform_pm1(int(n), seed(config, 100 * rep + s), lo, length)
        pos.append(a)
        q.append(b)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(np.asarray(sizes, dtype=np.int64))
    if not pos:
        return np.zeros((0, 3)), np.zeros(0), off
    return np.concatenate(pos, axis=0), np.concatenate(q), off


def rock_salt(n: int, length: float = 1.0):
    """One ion at the centre of every cell of an n^3 mesh over [0, length)^3, charge
    (-1)^(ix+iy+iz): the NaCl lattice with spacing length/n."""
    h = length / n
    idx = np.arange(n)
    ix, iy, iz = np.meshgrid(idx, idx, idx, indexing="ij")
    pos = np.stack([(ix + 0.5) * h, (iy + 0.5) * h, (iz + 0.5) * h], axis=-1).reshape(-1, 3)
    q = np.where(((ix + iy + iz) % 2) == 0, 1.0, -1.0).reshape(-1)
    return pos, q


def cell_centres(mesh, lo, length, s: int, fill: float = 1.0):
    """One particle at the centre of a random subset (fraction `fill`) of the cells,
    random charges in [-1, 1)."""
    g = rng(s)
    mesh = np.asarray(mesh)
    lo = np.asarray(lo, dtype=np.float64)
    length = np.asarray(length, dtype=np.float64)
    h = length / mesh
    ix, iy, iz = np.meshgrid(np.arange(mesh[0]), np.arange(mesh[1]), np.arange(mesh[2]), indexing="ij")
    c = np.stack([ix, iy, iz], axis=-1).reshape(-1, 3)
    keep = g.random(c.shape[0]) < fill
    c = c[keep]
    pos = lo + (c + 0.5) * h
    q = 2.0 * g.random(c.shape[0]) - 1.0
    return pos, q
