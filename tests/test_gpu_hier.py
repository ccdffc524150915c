"""GPU parity of the two-level PMMM (Sec. 5, hierarchical treatment; plans with
refine >= 2) against the oracle's cell-pair definition (oracle.pmmm_hier):

* FP64: fine multipoles to 1e-13 and the fine local expansions (L2L of the coarse
  locals plus the fine-level block convolution) to 1e-11 per order; forces,
  potentials and the energy to 1e-10, open and periodic, r = 2 and 4, c = 1 and 2;
* FP32 (SIMT matrix-product block M2L), split BF16 (tensor-core block M2L) and a
  high order (channel-major block spectra, per-wavevector M2L) within the
  tolerances of the one-level path;
* the launch configuration of the benchmark (N = 2^20, fine mesh 32^3, r = 4) on a
  seeded sample of cells;
* configurations the two-level path does not take are refused on the host.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = {p: 3e-6 * (1 + 0.25 * p) for p in range(0, 13)}
SPLITBF16_TOL = 2e-5


@pytest.fixture(scope="module")
def pk():
    import torch
    import paper_1409_5981_gb300 as pk
    pk.build()
    torch.cuda.set_device(0)
    return pk


def _t(a, dtype):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def _run(pk, cfg, pos, q):
    import torch
    dt = torch.float64 if cfg.precision == pk.FP64 else torch.float32
    plan = pk.Plan(cfg)
    phi, force, energy = plan.compute(_t(pos, dt), _t(q, dt), energy=True)
    torch.cuda.synchronize()
    return plan, phi.cpu().numpy().astype(np.float64), force.cpu().numpy().astype(np.float64), energy


def _oracle(cfg, pk, pos, q, target_cells=None, want_ml=False):
    alpha = cfg.ewald_alpha if cfg.ewald_alpha > 0 else None
    return oracle.pmmm_hier(pos, q, cfg.box_lo, cfg.box_len, cfg.mesh, cfg.p, cfg.refine, cfg.cutoff,
                            cfg.boundary == pk.PERIODIC, alpha=alpha, nmax=cfg.ewald_nmax or 5,
                            target_cells=target_cells, want_ml=want_ml)


@pytest.mark.parametrize("boundary", [0, 1])
def test_multipoles_and_locals_fp64(pk, boundary):
    pos, q = synth.uniform_pm1(3000, synth.seed(7, 1 + boundary))
    cfg = pk.Config(mesh=(8, 8, 8), p=4, boundary=boundary, precision=pk.FP64, refine=2)
    plan, *_ = _run(pk, cfg, pos, q)
    assert plan.info(pk.INFO_REFINE) == 2
    ref = _oracle(cfg, pk, pos, q, want_ml=True)
    M = plan.export(pk.EXPORT_MULTIPOLE)
    Mr = oracle.to_real_storage(ref["M"]).T
    assert np.abs(M - Mr).max() < 1e-13 * np.abs(Mr).max()
    Lg = plan.export(pk.EXPORT_LOCAL)
    Lr = oracle.to_real_storage(ref["L"]).T
    for l in range(cfg.p + 1):
        sl = slice(l * l, (l + 1) ** 2)
        err = np.abs(Lg[sl] - Lr[sl]).max() / np.abs(Lr[sl]).max()
        print(f"boundary={boundary} order {l}: fine locals max rel {err:.1e}")
        assert err < 1e-11, l
    plan.close()


@pytest.mark.parametrize("boundary", [0, 1])
@pytest.mark.parametrize("refine,cutoff,p", [(2, 1, 4), (4, 1, 4), (2, 2, 3)])
def test_full_fp64(pk, boundary, refine, cutoff, p):
    pos, q = synth.uniform_pm1(4096, synth.seed(7, 10 + 4 * refine + cutoff + boundary))
    if boundary == 1:
        q = q + 0.25 / 4096.0  # a charged periodic system exercises every coarse-level correction
    cfg = pk.Config(mesh=(16, 16, 16), p=p, cutoff=cutoff, boundary=boundary, precision=pk.FP64, refine=refine)
    plan, phi, force, energy = _run(pk, cfg, pos, q)
    ref = _oracle(cfg, pk, pos, q)
    rf = -(q[:, None] * ref["grad"])
    e_f, e_p = _rel(force, rf), _rel(phi, ref["phi"])
    print(f"fp64 two-level r={refine} c={cutoff} p={p} boundary={boundary}: force {e_f:.2e} phi {e_p:.2e}")
    assert e_f < FP64_TOL and e_p < FP64_TOL
    u = 0.5 * float((q * ref["phi"]).sum())
    assert abs(energy - u) < 1e-10 * abs(u)
    plan.close()


@pytest.mark.parametrize("boundary", [0, 1])
@pytest.mark.parametrize("precision,p,tol", [("fp32", 5, None), ("splitbf16", 7, SPLITBF16_TOL),
                                             ("fp32", 10, None)])
def test_fp32_paths(pk, boundary, precision, p, tol):
    pos, q = synth.uniform_pm1(8000, synth.seed(7, 30 + p + boundary))
    pos = pos.astype(np.float32).astype(np.float64)
    prec = pk.FP32 if precision == "fp32" else pk.FP32_SPLITBF16_M2L
    cfg = pk.Config(mesh=(16, 16, 16), p=p, boundary=boundary, precision=prec, refine=4)
    plan, phi, force, energy = _run(pk, cfg, pos, q)
    cells = synth.rng(702 + p).choice(16 ** 3, size=400, replace=False)
    ref = _oracle(cfg, pk, pos, q, target_cells=cells)
    sel = ~np.isnan(ref["phi"])
    rf = -(q[sel, None] * ref["grad"][sel])
    e_f, e_p = _rel(force[sel], rf), _rel(phi[sel], ref["phi"][sel])
    bound = FP32_TOL[p] if tol is None else tol
    print(f"{precision} two-level p={p} boundary={boundary}: force {e_f:.2e} phi {e_p:.2e} (bound {bound:.1e})")
    assert e_f < bound and e_p < bound
    plan.close()


def test_bench_configuration_sampled(pk):
    """N = 2^20 uniform +-1, periodic, fine mesh 32^3, r = 4 (coarse 8^3), p = 7, FP32:
    the launch configuration the benchmark times; the oracle checks sampled cells."""
    n = 1 << 20
    pos, q = synth.uniform_pm1(n, synth.seed(7, 0))
    pos = pos.astype(np.float32).astype(np.float64)
    cfg = pk.Config(mesh=(32, 32, 32), p=7, boundary=pk.PERIODIC, precision=pk.FP32, refine=4)
    plan, phi, force, energy = _run(pk, cfg, pos, q)
    cells = synth.rng(701).choice(32 ** 3, size=6, replace=False)
    ref = _oracle(cfg, pk, pos, q, target_cells=cells)
    sel = ~np.isnan(ref["phi"])
    rf = -(q[sel, None] * ref["grad"][sel])
    e_f, e_p = _rel(force[sel], rf), _rel(phi[sel], ref["phi"][sel])
    print(f"two-level 32^3 r=4 sampled {sel.sum()} particles: force {e_f:.2e} phi {e_p:.2e}")
    assert e_f < FP32_TOL[7] and e_p < FP32_TOL[7]
    plan.close()


def test_refusals(pk):
    import torch
    bad = [dict(mesh=(8, 8, 8), refine=3),                   # not a power of two
           dict(mesh=(8, 8, 12), refine=4),                  # mesh not divisible (and not a power of two)
           dict(mesh=(8, 8, 8), refine=4, boundary=1),       # periodic coarse mesh 2^3 < 2c + 1
           dict(mesh=(8, 8, 8), refine=32)]
    for kw in bad:
        with pytest.raises(pk.PmmmError):
            pk.Plan(pk.Config(p=3, **kw))
    with pytest.raises(pk.PmmmError):
        pk.Plan(pk.Config(mesh=(8, 8, 8), p=3, refine=-1))
    plan = pk.Plan(pk.Config(mesh=(16, 16, 16), p=3, precision=pk.FP32, refine=4))
    pos, q = synth.uniform_pm1(1000, synth.seed(7, 50))
    tp, tq = _t(pos, torch.float32), _t(q, torch.float32)
    with pytest.raises(pk.PmmmError):
        plan.compute_batched([500, 500], tp, tq)
    phi, force, _ = plan.compute_batched([1000], tp, tq)  # one system is the single-system path
    phi1, force1, _ = plan.compute(tp, tq)
    assert torch.equal(force, force1)
    plan.close()
    with pytest.raises(pk.PmmmError):
        pk.Surrogate(pk.Config(mesh=(8, 8, 8), p=3, boundary=pk.PERIODIC, precision=pk.FP32, refine=2), 10)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_refine8_long_block_transforms(pk, precision):
    """r = 8 (blocks of 32^3 fine cells, 24^3 kept outputs): the FP32 FFT inverse with
    one cell per block and the FP64 register-column inverse."""
    pos, q = synth.uniform_pm1(6000, synth.seed(7, 60))
    fp64 = precision == "fp64"
    if not fp64:
        pos = pos.astype(np.float32).astype(np.float64)
    cfg = pk.Config(mesh=(16, 16, 16), p=3, boundary=pk.OPEN, precision=pk.FP64 if fp64 else pk.FP32, refine=8)
    plan, phi, force, energy = _run(pk, cfg, pos, q)
    cells = synth.rng(703).choice(16 ** 3, size=300, replace=False)
    ref = _oracle(cfg, pk, pos, q, target_cells=cells)
    sel = ~np.isnan(ref["phi"])
    rf = -(q[sel, None] * ref["grad"][sel])
    e_f, e_p = _rel(force[sel], rf), _rel(phi[sel], ref["phi"][sel])
    bound = FP64_TOL if fp64 else FP32_TOL[3]
    print(f"{precision} two-level r=8: force {e_f:.2e} phi {e_p:.2e}")
    assert e_f < bound and e_p < bound
    plan.close()


def test_refine16_blocks_too_large_refused(pk):
    with pytest.raises(pk.PmmmError):
        pk.Plan(pk.Config(mesh=(32, 32, 32), p=3, boundary=pk.OPEN, precision=pk.FP32, refine=16))
