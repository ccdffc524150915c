"""Linear bound of the learned local-expansion correction, on the oracle side.

The learned correction maps the order-3 multipoles of a cell's 27 nearest cells
(27 x 16 = 432 numbers, real storage of App. A.7) to the difference between the
cell's order-10 and order-3 locals (121 numbers).  Before blaming training for a
network that gains nothing, this test asks how much of that difference the
27-cell window can carry at all: it fits the map by (lightly regularised) linear
least squares on oracle data of training systems and measures, on held-out
systems, the fraction of the target variance it explains (R^2) and the gain in
force accuracy of order 3 corrected by it, against plain order 10 (the
correction adds the far-field gradient of the predicted locals at each particle,
Eq. L2P with the order-one L2L of Eq. phigrad; near field and periodic
corrections are the same at both orders).

Pin of the pipeline: the exact targets (order-10 minus order-3 locals) used as
the correction reproduce the order-10 forces to rounding.

Data: periodic unit boxes, mesh 8^3, N = 4096 uniform +-1 charges (synth seeds
of the learned-correction configuration), 14 training and 2 held-out systems, 224
seeded target cells each (3136 training cells for 433 coefficients).
"""
import numpy as np

import oracle
import synth

MESH = 8
P_LO, P_HI = 3, 10
N = 4096
N_TRAIN, N_TEST = 14, 2
CELLS = 224


def _from_real_storage(x, p):
    """Real storage (App. A.7) -> complex full-index harmonics, X_l^-m = (-1)^m conj(X_l^m)."""
    out = np.zeros((p + 1) ** 2, dtype=np.complex128)
    for l in range(p + 1):
        out[oracle.hidx(l, 0)] = x[oracle.hidx(l, 0)]
        for m in range(1, l + 1):
            v = x[oracle.hidx(l, m)] + 1j * x[oracle.hidx(l, -m)]
            out[oracle.hidx(l, m)] = v
            out[oracle.hidx(l, -m)] = (-1) ** m * np.conj(v)
    return out


def _system(rep, green_lo, green_hi):
    pos, q = synth.uniform_pm1(N, synth.seed(5, 1000 + rep))
    cells = synth.rng(synth.seed(5, 2000 + rep)).choice(MESH ** 3, size=CELLS, replace=False)
    lo = oracle.pmmm(pos, q, (0, 0, 0), (1, 1, 1), (MESH,) * 3, P_LO, 1, True, target_cells=cells, want_ml=True,
                     green=green_lo)
    hi = oracle.pmmm(pos, q, (0, 0, 0), (1, 1, 1), (MESH,) * 3, P_HI, 1, True, target_cells=cells, want_ml=True,
                     green=green_hi)
    Mr = oracle.to_real_storage(lo["M"])  # (K, 16)
    Mg = Mr.reshape(MESH, MESH, MESH, 16)  # [z][y][x]
    X, Y = [], []
    for c in cells:
        ix, iy, iz = c % MESH, (c // MESH) % MESH, c // (MESH * MESH)
        f = []
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    f.append(Mg[(iz + dz) % MESH, (iy + dy) % MESH, (ix + dx) % MESH])
        X.append(np.concatenate(f))
        Lpad = np.zeros((P_HI + 1) ** 2, dtype=np.complex128)
        Lpad[: (P_LO + 1) ** 2] = lo["L"][c]
        Y.append(oracle.to_real_storage(hi["L"][c] - Lpad))
    return dict(pos=pos, q=q, cells=cells, lo=lo, hi=hi, X=np.array(X), Y=np.array(Y))


def _force_error(s, dY):
    """Relative RMS force error, against order 10, of order 3 plus the far-field
    gradient of the locals dY (real storage, one row per target cell)."""
    h = 1.0 / MESH
    st, cell, *_ = oracle.bin_particles(s["pos"], (0, 0, 0), (1, 1, 1), (MESH,) * 3, True)
    row = {int(c): i for i, c in enumerate(s["cells"])}
    num = den = 0.0
    for i in np.nonzero(~np.isnan(s["lo"]["phi"]))[0]:
        c = int(cell[i])
        ctr = (np.array([c % MESH, (c // MESH) % MESH, c // (MESH * MESH)]) + 0.5) * h
        r = s["pos"][i] - ctr
        r -= np.round(r)  # periodic wrap of the particle into its cell frame
        _, g = oracle.l2p(P_HI, _from_real_storage(dY[row[c]], P_HI), r)
        gc = s["lo"]["grad"][i] + g
        num += s["q"][i] ** 2 * ((gc - s["hi"]["grad"][i]) ** 2).sum()
        den += s["q"][i] ** 2 * (s["hi"]["grad"][i] ** 2).sum()
    return float(np.sqrt(num / den))


def test_linear_bound_of_the_27_cell_window():
    g_lo = oracle.green_table((0, 0, 0), (1, 1, 1), (MESH,) * 3, P_LO, 1, True)
    g_hi = oracle.green_table((0, 0, 0), (1, 1, 1), (MESH,) * 3, P_HI, 1, True)
    systems = [_system(r, g_lo, g_hi) for r in range(N_TRAIN + N_TEST)]
    train, test = systems[:N_TRAIN], systems[N_TRAIN:]

    # pin: the exact targets as the correction give the order-10 forces
    e_exact = _force_error(test[0], test[0]["Y"])
    assert e_exact < 1e-10, e_exact

    X = np.concatenate([s["X"] for s in train])
    Y = np.concatenate([s["Y"] for s in train])
    mu, sd = X.mean(0), X.std(0) + 1e-300
    ys = np.sqrt((Y ** 2).mean(0)) + 1e-300  # per-channel scale, as the network's target scaling
    A = np.hstack([(X - mu) / sd, np.ones((X.shape[0], 1))])
    lam = 1e-6 * np.trace(A.T @ A) / A.shape[1]
    W = np.linalg.solve(A.T @ A + lam * np.eye(A.shape[1]), A.T @ (Y / ys))

    def predict(Xn):
        return (np.hstack([(Xn - mu) / sd, np.ones((Xn.shape[0], 1))]) @ W) * ys

    Xt = np.concatenate([s["X"] for s in test])
    Yt = np.concatenate([s["Y"] for s in test])
    Yh = predict(Xt)
    r2_test = 1.0 - (((Yt - Yh) / ys) ** 2).sum() / (((Yt - Y.mean(0)) / ys) ** 2).sum()
    r2_train = 1.0 - (((Y - predict(X)) / ys) ** 2).sum() / (((Y - Y.mean(0)) / ys) ** 2).sum()
    e3 = np.mean([_force_error(s, np.zeros_like(s["Y"])) for s in test])
    elin = np.mean([_force_error(s, predict(s["X"])) for s in test])
    print(f"linear bound (27-cell window, p 3 -> 10, {X.shape[0]} training cells): R^2 train {r2_train:.3f}, "
          f"held-out {r2_test:.3f}; held-out force error plain p=3 {e3:.3e}, linear correction {elin:.3e} "
          f"(gain {e3 / elin:.3f})")
    assert np.isfinite(r2_test) and r2_test <= 1.0 and r2_train > 0.0
    assert e3 > 0.0 and elin > 0.0
