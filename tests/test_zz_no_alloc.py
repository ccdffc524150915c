"""pmmm_bin_sort_static: the allocation-free binning and cell sort for callers
that cannot call cudaMalloc (graph captures that must not allocate, memory pools
or host frameworks that own all device memory, loops that must never block in
the allocator).  Its cell offsets and stable permutation must be bit-identical
to those of the regular path (pmmm_compute, read back with pmmm_plan_export),
on two calls in a row that share the static scratch array.  This file is named
so that pytest collects it last."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    import torch
    import paper_1409_5981_gb300 as pk
    pk.build()
    torch.cuda.set_device(0)
    return pk


def _regular(pk, cfg, pos, q):
    import torch
    dt = torch.float64 if cfg.precision == pk.FP64 else torch.float32
    plan = pk.Plan(cfg)
    plan.compute(torch.tensor(pos, dtype=dt, device="cuda"), torch.tensor(q, dtype=dt, device="cuda"), energy=True)
    perm = plan.export(pk.EXPORT_PERM)
    cs = plan.export(pk.EXPORT_CELL_START)
    plan.close()
    return perm, cs


def _static(pk, cfg, pos):
    import torch
    dt = torch.float64 if cfg.precision == pk.FP64 else torch.float32
    n = pos.shape[0]
    K = int(np.prod(cfg.mesh))
    p = torch.tensor(pos, dtype=dt, device="cuda")
    perm = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")[:n]
    cs = torch.full((K + 1,), -7, dtype=torch.int32, device="cuda")
    st = pk.bin_sort_static(cfg, p, perm, cs)
    torch.cuda.synchronize()
    return st, perm.cpu().numpy(), cs.cpu().numpy()


@pytest.mark.parametrize("precision,boundary", [(1, 1), (0, 0), (1, 0)])
def test_static_sort_matches_regular_path_twice(pk, precision, boundary):
    cfg = pk.Config(box_lo=(-0.5, 0.0, 0.25), box_len=(1.0, 2.0, 0.5), mesh=(16, 8, 4), p=2, boundary=boundary,
                    precision=precision)
    for rep, n in enumerate((50000, 1237)):  # a second, smaller call after a larger one
        g = synth.rng(9100 + 10 * precision + 3 * boundary + rep)
        pos = np.asarray(cfg.box_lo) + g.random((n, 3)) * np.asarray(cfg.box_len)
        if boundary == pk.PERIODIC:
            pos[: n // 10] += np.round(g.standard_normal((n // 10, 3))) * np.asarray(cfg.box_len)
        if precision != pk.FP64:
            pos = pos.astype(np.float32).astype(np.float64)
        q = np.ones(n)
        st, perm, cs = _static(pk, cfg, pos)
        assert st == pk.OK
        rperm, rcs = _regular(pk, cfg, pos, q)
        assert np.array_equal(perm, rperm)
        assert np.array_equal(cs, rcs)


def test_static_sort_limits(pk):
    import torch
    cfg = pk.Config(mesh=(8, 8, 8), p=1, boundary=pk.PERIODIC, precision=pk.FP32)
    n = pk.STATIC_SORT_MAX_N + 1
    pos = torch.rand((n, 3), dtype=torch.float32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    cs = torch.empty(8 ** 3 + 1, dtype=torch.int32, device="cuda")
    assert pk.bin_sort_static(cfg, pos, perm, cs) == pk.ERR_UNSUPPORTED
    # at the limit it works, and an empty input gives an all-zero cell_start
    st = pk.bin_sort_static(cfg, pos[: pk.STATIC_SORT_MAX_N].contiguous(), perm, cs)
    assert st == pk.OK
    st = pk.bin_sort_static(cfg, pos[:0], perm, cs)
    assert st == pk.OK and int(cs.abs().sum()) == 0


def test_static_sort_at_the_limit_matches_regular_path(pk):
    """n = PMMM_STATIC_SORT_MAX_N fills every region of the static array to its sized
    bound; a non-cubic mesh of 2048 cells, FP32 and FP64 inputs, two calls in a row."""
    n = pk.STATIC_SORT_MAX_N
    for precision, boundary, mesh in ((pk.FP32, pk.PERIODIC, (16, 8, 16)), (pk.FP64, pk.OPEN, (32, 4, 16))):
        cfg = pk.Config(box_lo=(0.0, -1.0, 0.5), box_len=(2.0, 1.0, 1.5), mesh=mesh, p=1, boundary=boundary,
                        precision=precision)
        for rep in range(2):
            g = synth.rng(9300 + 7 * precision + rep)
            pos = np.asarray(cfg.box_lo) + g.random((n, 3)) * np.asarray(cfg.box_len)
            if precision != pk.FP64:
                pos = pos.astype(np.float32).astype(np.float64)
            st, perm, cs = _static(pk, cfg, pos)
            assert st == pk.OK
            rperm, rcs = _regular(pk, cfg, pos, np.ones(n))
            assert np.array_equal(perm, rperm)
            assert np.array_equal(cs, rcs)


def test_static_sort_wrapper_rejects_bad_tensors(pk):
    """The binding checks dtype, shape, sizes, contiguity and device before any launch."""
    import torch
    cfg = pk.Config(mesh=(8, 8, 8), p=1, boundary=pk.PERIODIC, precision=pk.FP64)
    n, K = 1000, 8 ** 3
    pos = torch.rand((n, 3), dtype=torch.float64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    cs = torch.empty(K + 1, dtype=torch.int32, device="cuda")
    bad = [
        (pos.float(), perm, cs),                                   # FP32 positions under an FP64 config
        (pos.reshape(-1)[: 2 * n].reshape(n, 2), perm, cs),       # wrong shape
        (pos, perm[: n - 1], cs),                                  # short perm
        (pos, perm.long(), cs),                                    # wrong index type
        (pos, perm, cs[:K]),                                       # short cell_start
        (pos.t().contiguous().t(), perm, cs),                      # not contiguous
        (pos.cpu(), perm, cs),                                     # host tensor
    ]
    for a, b, c in bad:
        with pytest.raises(ValueError):
            pk.bin_sort_static(cfg, a, b, c)
    assert pk.bin_sort_static(cfg, pos, perm, cs) == pk.OK
