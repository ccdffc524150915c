"""GPU parity of the batched form (pmmm_compute_batched): many independent systems
on one plan, laid side by side as one mesh, with the per-wavevector M2L done as one
complex matrix product over all systems.

Each system's potentials, forces and energy must equal those of pmmm_compute on
that system alone -- the two paths differ only in the M2L accumulation order, so
FP64 agrees to 1e-12 relative RMS and FP32 within the FP32 tolerance -- and, at
sizes the oracle finishes quickly, the FP64 oracle's PMMM of each system.  Cell
binning is bit-exact: the cell offsets of system s are those of its own plan,
shifted by its first particle."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import force_errors, green, sample_cells

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
BATCH_VS_SINGLE_FP64 = 1e-12
FP32_TOL = {p: 3e-6 * (1 + 0.25 * p) for p in range(0, 13)}
# relative RMS force / potential error bound of the split-BF16 tensor-core M2L against
# the FP32 path: each M2L product carries <= 3 * 2^-18 relative error (hi + lo
# representation of both operands, lo * lo dropped), i.e. ~1.1e-5 per term; the
# far field is a fraction of each force, so the force error stays below 2e-5
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


def _dt(pk, cfg):
    import torch
    return torch.float64 if cfg.precision == pk.FP64 else torch.float32


def _systems(pk, cfg, sizes, config, wrap=False):
    pos, q, off = synth.batched_uniform_pm1(sizes, config, lo=cfg.box_lo, length=cfg.box_len)
    if wrap and pos.shape[0]:
        g = synth.rng(synth.seed(config, 99))
        k = pos.shape[0] // 10
        pos[:k] += np.round(g.standard_normal((k, 3))) * np.asarray(cfg.box_len)
    if cfg.precision != pk.FP64:
        pos = pos.astype(np.float32).astype(np.float64)
    return pos, q, off


def _batched(pk, cfg, pos, q, off):
    import torch
    plan = pk.Plan(cfg)
    dt = _dt(pk, cfg)
    phi, force, e = plan.compute_batched(np.diff(off), _t(pos, dt), _t(q, dt), energies=True)
    torch.cuda.synchronize()
    return plan, phi.double().cpu().numpy(), force.double().cpu().numpy(), e


def _single(pk, cfg, pos, q):
    import torch
    plan = pk.Plan(cfg)
    dt = _dt(pk, cfg)
    phi, force, e = plan.compute(_t(pos, dt), _t(q, dt), energy=True)
    cs = plan.export(pk.EXPORT_CELL_START)
    perm = plan.export(pk.EXPORT_PERM)
    plan.close()
    return phi.double().cpu().numpy(), force.double().cpu().numpy(), e, cs, perm


def _check_against_single(pk, cfg, sizes, config, wrap=False):
    pos, q, off = _systems(pk, cfg, sizes, config, wrap)
    plan, phi, force, energies = _batched(pk, cfg, pos, q, off)
    K = int(np.prod(cfg.mesh))
    B = len(sizes)
    cs_all = plan.export(pk.EXPORT_CELL_START)
    perm_all = plan.export(pk.EXPORT_PERM)
    assert cs_all.shape == (B * K + 1,)
    tol = BATCH_VS_SINGLE_FP64 if cfg.precision == pk.FP64 else FP32_TOL[cfg.p]
    worst = 0.0
    for s in range(B):
        a, b = off[s], off[s + 1]
        assert cs_all[s * K] == a
        if b == a:
            continue
        sphi, sforce, se, scs, sperm = _single(pk, cfg, pos[a:b], q[a:b])
        assert np.array_equal(cs_all[s * K: (s + 1) * K + 1], scs + a), s
        assert np.array_equal(perm_all[a:b], sperm + a), s
        ef, ep = _rel(force[a:b], sforce), _rel(phi[a:b], sphi)
        eu = abs(energies[s] - se) / max(abs(se), 1e-300)
        worst = max(worst, ef, ep)
        assert ef < tol and ep < tol, (s, ef, ep)
        if cfg.precision == pk.FP64:
            assert eu < 1e-12, (s, eu)
        else:
            # U = 1/2 sum q phi: by Cauchy-Schwarz the energies of two evaluations differ
            # by at most 1/2 |q| |phi_a - phi_b| (the potentials checked above), plus the
            # FP32 rounding of the per-item partial sums (~1e-6 of 1/2 sum |q phi|); the
            # energy of a neutral system cancels strongly, so a relative bound on U alone
            # would measure that cancellation rather than the arithmetic
            du = abs(energies[s] - se)
            bound = 0.5 * np.linalg.norm(q[a:b]) * np.linalg.norm(phi[a:b] - sphi) \
                + 1e-6 * 0.5 * np.abs(q[a:b] * sphi).sum()
            assert du <= bound, (s, du, bound, eu)
    print(f"batched vs single ({B} systems, p={cfg.p}, prec={cfg.precision}, bnd={cfg.boundary}): worst {worst:.2e}")
    plan.close()


@pytest.mark.parametrize("p", [2, 7])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("boundary", [0, 1])
def test_batched_matches_single_systems(pk, p, precision, boundary):
    """Uneven systems, including an empty one and a lone particle, across several
    sort tiles with ragged tails."""
    cfg = pk.Config(mesh=(8, 8, 8), p=p, boundary=boundary, precision=precision)
    _check_against_single(pk, cfg, [3001, 0, 1, 517, 4096, 2], 40 + 10 * p + 2 * precision + boundary,
                          wrap=boundary == pk.PERIODIC)


@pytest.mark.parametrize("p,precision", [(10, 0), (12, 1), (11, 1), (9, 0)])
def test_batched_high_order_paths(pk, p, precision):
    """Orders whose matrix A~(k) does not fit in shared memory take the per-wavevector
    kernel over all systems (FP64 p = 10, FP32 p = 12); FP32 p = 11 and FP64 p = 9 are
    the largest that take the matrix product."""
    cfg = pk.Config(mesh=(4, 4, 4), p=p, boundary=pk.PERIODIC, precision=precision, ewald_nmax=3)
    _check_against_single(pk, cfg, [700, 1200, 33, 901, 64], 60 + p + precision)


def test_batched_many_systems_tiles(pk):
    """More systems than one block of the matrix product holds (the system tiles and
    their ragged last tile), FP32 p = 7 on a 4^3 mesh."""
    sizes = synth.batched_sizes(70, synth.seed(4, 7), lo_exp=6, hi_exp=9)
    cfg = pk.Config(mesh=(4, 4, 4), p=7, boundary=pk.PERIODIC, precision=pk.FP32)
    _check_against_single(pk, cfg, list(sizes), 47)


@pytest.mark.parametrize("boundary", [0, 1])
def test_batched_fp64_vs_oracle(pk, boundary):
    """Each system of a batch against the FP64 oracle PMMM of that system."""
    cfg = pk.Config(mesh=(8, 8, 8), p=5, boundary=boundary, precision=pk.FP64, ewald_nmax=4)
    sizes = [900, 1500, 2, 1100]
    pos, q, off = _systems(pk, cfg, sizes, 48 + boundary)
    plan, phi, force, energies = _batched(pk, cfg, pos, q, off)
    for s in range(len(sizes)):
        a, b = off[s], off[s + 1]
        ref = oracle.pmmm(pos[a:b], q[a:b], cfg.box_lo, cfg.box_len, cfg.mesh, cfg.p, cfg.cutoff,
                          boundary == pk.PERIODIC, nmax=cfg.ewald_nmax)
        rf = -(q[a:b, None] * ref["grad"])
        ef, ep = _rel(force[a:b], rf), _rel(phi[a:b], ref["phi"])
        eu = abs(energies[s] - 0.5 * (q[a:b] * ref["phi"]).sum()) / abs(0.5 * (q[a:b] * ref["phi"]).sum())
        assert ef < FP64_TOL and ep < FP64_TOL and eu < FP64_TOL, (s, ef, ep, eu)
    if boundary == pk.PERIODIC:
        corr = plan.export(pk.EXPORT_CORR)
        assert corr.shape == (len(sizes), 8)
        for s in range(len(sizes)):
            a, b = off[s], off[s + 1]
            assert abs(corr[s, 0] - q[a:b].sum()) < 1e-12
    plan.close()


def test_batched_host_api_and_reuse(pk):
    """Host arrays give the device results bit for bit; a plan reused with other
    offsets, then for one system, gives what fresh plans give."""
    import torch
    cfg = pk.Config(mesh=(8, 8, 8), p=4, boundary=pk.PERIODIC, precision=pk.FP32)
    pos, q, off = _systems(pk, cfg, [1000, 2500, 10], 50)
    plan = pk.Plan(cfg)
    dt = torch.float32
    phi_d, force_d, e_d = plan.compute_batched(np.diff(off), _t(pos, dt), _t(q, dt), energies=True)
    phi_h, force_h, e_h = plan.compute_batched_host(np.diff(off), pos.astype(np.float32), q.astype(np.float32))
    assert np.array_equal(phi_d.cpu().numpy(), phi_h) and np.array_equal(force_d.cpu().numpy(), force_h)
    assert np.array_equal(e_d, e_h)
    # other offsets on the same plan
    pos2, q2, off2 = _systems(pk, cfg, [3000, 7, 400, 1], 51)
    phi2, force2, e2 = plan.compute_batched(np.diff(off2), _t(pos2, dt), _t(q2, dt), energies=True)
    fresh, fphi2, fforce2, fe2 = _batched(pk, cfg, pos2, q2, off2)
    fresh.close()
    assert np.array_equal(phi2.double().cpu().numpy(), fphi2) and np.array_equal(force2.double().cpu().numpy(), fforce2)
    # one system on the grown plan
    phi1, force1, e1 = plan.compute(_t(pos2[:3000], dt), _t(q2[:3000], dt), energy=True)
    sphi, sforce, se, _, _ = _single(pk, cfg, pos2[:3000], q2[:3000])
    assert np.array_equal(phi1.double().cpu().numpy(), sphi) and np.array_equal(force1.double().cpu().numpy(), sforce)
    assert plan.info(pk.INFO_SYSTEMS) == 1
    plan.close()


def test_batched_input_errors(pk):
    import ctypes
    import torch
    cfg = pk.Config(mesh=(4, 4, 4), p=2, boundary=pk.OPEN, precision=pk.FP64)
    plan = pk.Plan(cfg)
    lib = pk._lib()
    pos = torch.rand((10, 3), dtype=torch.float64, device="cuda")
    q = torch.ones(10, dtype=torch.float64, device="cuda")
    out = torch.empty((10, 3), dtype=torch.float64, device="cuda")

    def call(off, nsys=None):
        off = np.asarray(off, dtype=np.int64)
        return lib.pmmm_compute_batched(plan._h, len(off) - 1 if nsys is None else nsys,
                                        ctypes.c_void_p(off.ctypes.data), ctypes.c_void_p(pos.data_ptr()),
                                        ctypes.c_void_p(q.data_ptr()), None, ctypes.c_void_p(out.data_ptr()), None)
    assert call([1, 5, 10]) == pk.ERR_INVALID_ARG      # offsets[0] != 0
    assert call([0, 6, 5]) == pk.ERR_INVALID_ARG       # decreasing
    assert call([0, 10], nsys=0) == pk.ERR_INVALID_ARG
    assert call([0, 10], nsys=pk.MAX_SYSTEMS + 1) == pk.ERR_INVALID_ARG
    assert call([0, 4, 10]) == pk.OK
    torch.cuda.synchronize()
    # a particle outside the open box in the second system
    pos[7, 1] = 1.5
    e = np.zeros(2)
    off = np.array([0, 4, 10], dtype=np.int64)
    st = lib.pmmm_compute_batched(plan._h, 2, ctypes.c_void_p(off.ctypes.data), ctypes.c_void_p(pos.data_ptr()),
                                  ctypes.c_void_p(q.data_ptr()), None, ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(e.ctypes.data))
    assert st == pk.ERR_OUT_OF_BOX
    assert plan.status() == pk.OK   # the flag was cleared
    plan.close()


def test_batched_config4_sampled(pk):
    """64 periodic systems, N log-uniform in [2^14, 2^18] (even), uniform +-1 neutral,
    mesh 32^3, p = 7, FP32, in the launch configuration the benchmark times: three
    systems against their own single-system evaluation on every particle, and the
    smallest against the oracle on sampled cells."""
    sizes = synth.batched_sizes(64, synth.seed(4, 0))
    cfg = pk.Config(mesh=(32, 32, 32), p=7, boundary=pk.PERIODIC, precision=pk.FP32)
    pos, q, off = _systems(pk, cfg, sizes, 4)
    plan, phi, force, energies = _batched(pk, cfg, pos, q, off)
    plan.close()
    smallest, largest = int(np.argmin(sizes)), int(np.argmax(sizes))
    for s in (smallest, largest, 17):
        a, b = off[s], off[s + 1]
        sphi, sforce, se, _, _ = _single(pk, cfg, pos[a:b], q[a:b])
        ef, ep = _rel(force[a:b], sforce), _rel(phi[a:b], sphi)
        print(f"config4 system {s} (N={b - a}) batched vs single: force {ef:.2e} phi {ep:.2e}")
        assert ef < FP32_TOL[7] and ep < FP32_TOL[7]
        # the Cauchy-Schwarz energy bound of _check_against_single
        bound = 0.5 * np.linalg.norm(q[a:b]) * np.linalg.norm(phi[a:b] - sphi) \
            + 1e-6 * 0.5 * np.abs(q[a:b] * sphi).sum()
        assert abs(energies[s] - se) <= bound
    G = green(cfg.box_lo, cfg.box_len, cfg.mesh, cfg.p, cfg.cutoff, True)
    a, b = off[smallest], off[smallest + 1]
    counts = np.bincount(_cells_of(pos[a:b], cfg), minlength=32 ** 3)
    cells = sample_cells(counts, cfg.mesh, 208)
    ref = oracle.pmmm(pos[a:b], q[a:b], cfg.box_lo, cfg.box_len, cfg.mesh, cfg.p, cfg.cutoff, True,
                      target_cells=cells, green=G)
    sel = ~np.isnan(ref["phi"])
    ef, emax, e99 = force_errors(force[a:b][sel], -(q[a:b][sel, None] * ref["grad"][sel]))
    ep = _rel(phi[a:b][sel], ref["phi"][sel])
    print(f"config4 system {smallest} sampled {len(cells)} cells, {sel.sum()} particles vs oracle: force rms {ef:.2e} "
          f"(per particle max {emax:.2e}, p99 {e99:.2e}) phi {ep:.2e}")
    assert ef < FP32_TOL[7] and ep < FP32_TOL[7]


def _cells_of(pos, cfg):
    """Cell id of each particle (for choosing sampled cells only: oracle binning)."""
    st, cell, *_ = oracle.bin_particles(pos, cfg.box_lo, cfg.box_len, cfg.mesh, cfg.boundary == 1)
    assert st == 0
    return cell


def test_batched_config4_splitbf16_sampled_vs_oracle(pk):
    """The benchmarked batched workload with the tensor-core M2L: 64 periodic systems, N
    log-uniform in [2^14, 2^18], mesh 32^3, p = 7, split BF16 (PMMM_INFO_M2L_ARITH says
    the tensor cores ran).  The smallest and the largest system against the oracle PMMM
    on 32 sampled cells each (the four most crowded, eight on the box faces, the rest
    random), within SPLITBF16_TOL."""
    import torch
    sizes = synth.batched_sizes(64, synth.seed(4, 0))
    cfg = pk.Config(mesh=(32, 32, 32), p=7, boundary=pk.PERIODIC, precision=pk.FP32_SPLITBF16_M2L)
    pos, q, off = _systems(pk, cfg, sizes, 4)
    plan, phi, force, energies = _batched(pk, cfg, pos, q, off)
    assert plan.info(pk.INFO_M2L_ARITH) == pk.M2L_ARITH_SPLITBF16_TC
    plan.close()
    G = green(cfg.box_lo, cfg.box_len, cfg.mesh, cfg.p, cfg.cutoff, True)
    for s_ in (int(np.argmin(sizes)), int(np.argmax(sizes))):
        a, b = off[s_], off[s_ + 1]
        counts = np.bincount(_cells_of(pos[a:b], cfg), minlength=32 ** 3)
        cells = sample_cells(counts, cfg.mesh, 210 + s_)
        ref = oracle.pmmm(pos[a:b], q[a:b], cfg.box_lo, cfg.box_len, cfg.mesh, cfg.p, cfg.cutoff, True,
                          target_cells=cells, green=G)
        sel = ~np.isnan(ref["phi"])
        ef, emax, e99 = force_errors(force[a:b][sel], -(q[a:b][sel, None] * ref["grad"][sel]))
        ep = _rel(phi[a:b][sel], ref["phi"][sel])
        print(f"config4 split-BF16 system {s_} (N={b - a}) sampled {len(cells)} cells, {sel.sum()} particles vs "
              f"oracle: force rms {ef:.2e} (per particle max {emax:.2e}, p99 {e99:.2e}) phi {ep:.2e}")
        assert len(cells) == 32 and ef < SPLITBF16_TOL and ep < SPLITBF16_TOL


def test_m2l_arithmetic_is_reported(pk):
    """PMMM_INFO_M2L_ARITH names the M2L that ran: the tensor cores only for batched
    split-BF16 evaluations with p <= 7; FP32 SIMT for one system or p > 7."""
    import torch
    sizes = [900, 1300, 700]
    for p, prec, batched, want in ((3, pk.FP32_SPLITBF16_M2L, True, pk.M2L_ARITH_SPLITBF16_TC),
                                   (3, pk.FP32_SPLITBF16_M2L, False, pk.M2L_ARITH_FP32_SIMT),
                                   (8, pk.FP32_SPLITBF16_M2L, True, pk.M2L_ARITH_FP32_SIMT),
                                   (3, pk.FP32, True, pk.M2L_ARITH_FP32_SIMT),
                                   (3, pk.FP64, False, pk.M2L_ARITH_FP64_SIMT)):
        cfg = pk.Config(mesh=(8, 8, 8), p=p, boundary=pk.PERIODIC, precision=prec, ewald_nmax=3)
        pos, q, off = _systems(pk, cfg, sizes, 58)
        dt = _dt(pk, cfg)
        plan = pk.Plan(cfg)
        assert plan.info(pk.INFO_M2L_ARITH) == -1
        if batched:
            plan.compute_batched(np.diff(off), _t(pos, dt), _t(q, dt))
        else:
            plan.compute(_t(pos[: off[1]], dt), _t(q[: off[1]], dt))
        torch.cuda.synchronize()
        assert plan.info(pk.INFO_M2L_ARITH) == want, (p, prec, batched)
        plan.close()


def test_batched_graph_replay(pk):
    """The CUDA-graph form gives the plain batched results bit for bit, on replay with
    new input values in the same buffers, and after a capture for other offsets."""
    import torch
    cfg = pk.Config(mesh=(8, 8, 8), p=5, boundary=pk.PERIODIC, precision=pk.FP32)
    stream = torch.cuda.Stream()
    plan = pk.Plan(cfg, stream=stream)
    dt = torch.float32
    pos, q, off = _systems(pk, cfg, [2000, 5, 3100], 52)
    counts = np.diff(off)
    tp, tq = _t(pos, dt), _t(q, dt)
    phi = torch.empty(len(q), dtype=dt, device="cuda")
    force = torch.empty((len(q), 3), dtype=dt, device="cuda")
    torch.cuda.synchronize()
    plan.compute_batched_graph(counts, tp, tq, phi, force, energies=True)      # capture + launch
    a_phi, a_force = phi.cpu().numpy().copy(), force.cpu().numpy().copy()
    ref, rphi, rforce, re = _batched(pk, cfg, pos, q, off)
    ref.close()
    assert np.array_equal(a_phi.astype(np.float64), rphi) and np.array_equal(a_force.astype(np.float64), rforce)
    # new values in the same buffers: replay
    pos2, q2, _ = _systems(pk, cfg, [2000, 5, 3100], 53)
    with torch.cuda.stream(stream):
        tp.copy_(_t(pos2, dt))
        tq.copy_(_t(q2, dt))
    stream.synchronize()
    _, _, e2 = plan.compute_batched_graph(counts, tp, tq, phi, force, energies=True)
    ref, rphi2, rforce2, re2 = _batched(pk, cfg, pos2, q2, off)
    ref.close()
    assert np.array_equal(phi.double().cpu().numpy(), rphi2) and np.array_equal(force.double().cpu().numpy(), rforce2)
    assert np.array_equal(e2, re2)
    # other offsets: a new capture
    counts3 = np.array([1000, 4105])
    _, _, e3 = plan.compute_batched_graph(counts3, tp, tq, phi, force, energies=True)
    off3 = np.concatenate([[0], np.cumsum(counts3)])
    ref, rphi3, rforce3, re3 = _batched(pk, cfg, pos2, q2, off3)
    ref.close()
    assert np.array_equal(phi.double().cpu().numpy(), rphi3) and np.array_equal(e3, re3)
    plan.close()


@pytest.mark.parametrize("p", [2, 5, 7])
@pytest.mark.parametrize("boundary", [0, 1])
def test_batched_splitbf16_tensor_core_m2l(pk, p, boundary):
    """The batched M2L on the tensor cores (precision FP32_SPLITBF16_M2L, p <= 7):
    locals of every system against the FP32 batched path, and forces against the
    FP64 path, over two system tiles (70 systems: 64 + a ragged 6)."""
    import torch
    sizes = list(synth.batched_sizes(70, synth.seed(4, 8 + boundary), lo_exp=7, hi_exp=10))
    sizes[3] = 0
    res = {}
    for prec in (pk.FP32_SPLITBF16_M2L, pk.FP32, pk.FP64):
        cfg = pk.Config(mesh=(8, 8, 8), p=p, boundary=boundary, precision=prec, ewald_nmax=4)
        pos, q, off = _systems(pk, cfg if prec != pk.FP64 else pk.Config(precision=pk.FP32), sizes, 54 + boundary)
        plan, phi, force, e = _batched(pk, cfg, pos, q, off)
        res[prec] = (phi, force, e, plan.export(pk.EXPORT_LOCAL))
        plan.close()
    L_tc, L_32 = res[pk.FP32_SPLITBF16_M2L][3], res[pk.FP32][3]
    eL = float(np.abs(L_tc - L_32).max() / np.abs(L_32).max())
    ef = _rel(res[pk.FP32_SPLITBF16_M2L][1], res[pk.FP64][1])
    ef32 = _rel(res[pk.FP32][1], res[pk.FP64][1])
    ep = _rel(res[pk.FP32_SPLITBF16_M2L][0], res[pk.FP64][0])
    print(f"split-BF16 M2L p={p} bnd={boundary}: locals vs FP32 {eL:.2e}; force vs FP64 {ef:.2e} "
          f"(FP32 path {ef32:.2e}), phi {ep:.2e}")
    assert eL < 1e-4
    assert ef < SPLITBF16_TOL and ep < SPLITBF16_TOL


def test_autotune_choices_are_equivalent(pk):
    """pmmm_plan_autotune picks a near-field kernel (cell items with or without the far
    field beside them, or one thread per target) and a tensor-core M2L tile by timing;
    whatever it picks, the results agree with the untuned plan to rounding, and the
    chosen configuration reproduces itself bit for bit."""
    import torch
    cfg = pk.Config(mesh=(8, 8, 8), p=5, boundary=pk.PERIODIC, precision=pk.FP32_SPLITBF16_M2L)
    pos, q, off = _systems(pk, cfg, [1500, 700, 2600, 40, 900], 56)
    counts = np.diff(off)
    tp, tq = _t(pos, torch.float32), _t(q, torch.float32)
    base = pk.Plan(cfg)
    phi0, f0, e0 = base.compute_batched(counts, tp, tq, energies=True)
    plan = pk.Plan(cfg)
    near, tile = plan.autotune(counts, tp, tq, reps=2)
    assert near in (pk.NEAR_CELL_ITEMS, pk.NEAR_PER_TARGET, pk.NEAR_CELL_ITEMS_SPLIT) and tile in (32, 64)
    phi1, f1, e1 = plan.compute_batched(counts, tp, tq, energies=True)
    phi2, f2, e2 = plan.compute_batched(counts, tp, tq, energies=True)
    assert torch.equal(phi1, phi2) and torch.equal(f1, f2) and np.array_equal(e1, e2)
    a, b = f1.double().cpu().numpy(), f0.double().cpu().numpy()
    assert _rel(a, b) < 2e-6
    print(f"autotune: near-field kernel {near}, M2L tile {tile}")
    base.close()
    plan.close()


def test_batched_degenerate_batches(pk):
    """A batch of one system equals pmmm_compute bit for bit; a batch of empty systems
    gives zero energies and no particles."""
    import torch
    cfg = pk.Config(mesh=(8, 8, 8), p=4, boundary=pk.PERIODIC, precision=pk.FP32)
    pos, q, off = _systems(pk, cfg, [2345], 57)
    plan = pk.Plan(cfg)
    phi_b, f_b, e_b = plan.compute_batched([2345], _t(pos, torch.float32), _t(q, torch.float32), energies=True)
    phi_s, f_s, e_s = plan.compute(_t(pos, torch.float32), _t(q, torch.float32), energy=True)
    assert torch.equal(phi_b, phi_s) and torch.equal(f_b, f_s) and e_b[0] == e_s
    empty = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    phi0, f0, e0 = plan.compute_batched([0, 0, 0], empty, torch.zeros(0, dtype=torch.float32, device="cuda"),
                                        energies=True)
    assert phi0.numel() == 0 and np.array_equal(e0, np.zeros(3))
    plan.close()
