"""Helpers of the full-size parity tests: the choice of sampled target cells, the
error report, and a per-process cache of the oracle's Green-function tables (the
set-up step of Sec. 2.1, shared by every test that uses the same geometry).

Nothing here computes any part of the method: the cell choice uses only the
particle counts per cell, the error report compares two given force arrays, and
the cached tables come from oracle.green_table."""
import numpy as np

import oracle
import synth

_GREEN = {}


def green(lo, length, mesh, p, c, periodic, alpha=None, nmax=5):
    """oracle.green_table for this geometry, computed once per process."""
    key = (tuple(map(float, lo)), tuple(map(float, length)), tuple(map(int, mesh)), int(p), int(c), bool(periodic),
           None if alpha is None else float(alpha), int(nmax))
    if key not in _GREEN:
        _GREEN.clear()  # one table at a time: a 64^3, p = 7 table is close to 1 GB
        _GREEN[key] = oracle.green_table(lo, length, mesh, p, c, periodic, alpha=alpha, nmax=nmax)
    return _GREEN[key]


def sample_cells(counts, mesh, seed, n=32, crowded=4, faces=8):
    """n distinct target cells: the `crowded` most populated cells, `faces` random
    cells on the box faces (some index 0 or n-1 on an axis; the first is the corner
    cell 0), the rest random among the non-empty cells."""
    counts = np.asarray(counts)
    K = counts.shape[0]
    nx, ny, nz = (int(v) for v in mesh)
    g = synth.rng(seed)
    chosen = list(np.argsort(counts, kind="stable")[::-1][:crowded])
    idx = np.arange(K)
    ix, iy, iz = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    on_face = (ix == 0) | (ix == nx - 1) | (iy == 0) | (iy == ny - 1) | (iz == 0) | (iz == nz - 1)
    face_cells = [0] + list(g.permutation(np.nonzero(on_face)[0]))
    for c in face_cells:
        if len(chosen) >= crowded + faces:
            break
        if c not in chosen:
            chosen.append(int(c))
    rest = [int(c) for c in g.permutation(np.nonzero(counts > 0)[0]) if c not in chosen]
    chosen += rest[: max(0, n - len(chosen))]
    return np.array(chosen[:n], dtype=np.int64)


def force_errors(f, ref):
    """(relative RMS error, largest per-particle relative error, its 99th percentile)
    of forces f against ref, both (m, 3)."""
    f = np.asarray(f, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = np.sqrt(((f - ref) ** 2).sum(1))
    r = np.sqrt((ref ** 2).sum(1))
    rms = float(np.sqrt((d ** 2).sum() / max((r ** 2).sum(), 1e-300)))
    per = d / np.maximum(r, 1e-300)
    return rms, float(per.max()) if per.size else 0.0, float(np.percentile(per, 99)) if per.size else 0.0
