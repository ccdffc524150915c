"""Launch form of pmmm_compute: from the second identical call in a row on, the
evaluation is launched as a CUDA graph of the plain launch sequence.  Its results
must equal those of the plain sequence bit for bit: on the capturing call, on
replays that read new input values from the same buffers, after a workspace
reallocation (which forces a new capture), on the legacy default stream and on a
created stream, for one- and two-level plans; the batched graph call works on the
legacy default stream too."""
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


def _plain(pk, cfg, pos, q):
    """Results of the plain launch sequence: stage timing keeps every call uncaptured."""
    import torch
    plan = pk.Plan(cfg)
    plan.set_timing(True)
    tp = torch.tensor(pos, dtype=torch.float32, device="cuda")
    tq = torch.tensor(q, dtype=torch.float32, device="cuda")
    phi, force, _ = plan.compute(tp, tq, energy=True)
    out = phi.cpu().numpy().copy(), force.cpu().numpy().copy()
    plan.close()
    return out


@pytest.mark.parametrize("refine", [0, 2])
@pytest.mark.parametrize("own_stream", [False, True])
def test_single_call_graph(pk, own_stream, refine):
    import torch
    n = 3000
    cfg = pk.Config(mesh=(8, 8, 8), p=5, boundary=pk.PERIODIC, precision=pk.FP32, refine=refine)
    pos, q = synth.uniform_pm1(n, synth.seed(7, 1))
    pos, q = pos.astype(np.float32), q.astype(np.float32)
    pos2, q2 = synth.uniform_pm1(n, synth.seed(7, 2))
    pos2, q2 = pos2.astype(np.float32), q2.astype(np.float32)
    ref1, ref2 = _plain(pk, cfg, pos, q), _plain(pk, cfg, pos2, q2)

    stream = torch.cuda.Stream() if own_stream else torch.cuda.current_stream()
    tp = torch.tensor(pos, device="cuda")
    tq = torch.tensor(q, device="cuda")
    phi = torch.empty(n, dtype=torch.float32, device="cuda")
    force = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    plan = pk.Plan(cfg, stream)

    def call():
        assert plan.compute_raw(n, tp.data_ptr(), tq.data_ptr(), phi.data_ptr(), force.data_ptr()) == 0
        stream.synchronize()
        assert plan.status() == 0
        return phi.cpu().numpy().copy(), force.cpu().numpy().copy()

    # plain, capture + launch, replay
    for k in range(3):
        a_phi, a_force = call()
        assert np.array_equal(a_phi, ref1[0]) and np.array_equal(a_force, ref1[1]), f"call {k}"
    # new values in the same buffers: the replay reads them
    tp.copy_(torch.tensor(pos2, device="cuda"))
    tq.copy_(torch.tensor(q2, device="cuda"))
    torch.cuda.synchronize()
    a_phi, a_force = call()
    assert np.array_equal(a_phi, ref2[0]) and np.array_equal(a_force, ref2[1])
    # a larger reservation moves the particle workspace: plain call, then a new capture
    plan.reserve(4 * n)
    for k in range(3):
        a_phi, a_force = call()
        assert np.array_equal(a_phi, ref2[0]) and np.array_equal(a_force, ref2[1]), f"after reserve, call {k}"
    plan.close()


def test_batched_graph_default_stream(pk):
    import torch
    cfg = pk.Config(mesh=(8, 8, 8), p=4, boundary=pk.PERIODIC, precision=pk.FP32)
    counts = np.array([1200, 0, 700])
    n = int(counts.sum())
    pos, q = synth.uniform_pm1(n, synth.seed(7, 3))
    tp = torch.tensor(pos.astype(np.float32), device="cuda")
    tq = torch.tensor(q.astype(np.float32), device="cuda")
    plain = pk.Plan(cfg)
    rphi, rforce, re = plain.compute_batched(counts, tp, tq, energies=True)
    rphi, rforce = rphi.cpu().numpy(), rforce.cpu().numpy()
    plain.close()
    plan = pk.Plan(cfg)  # torch's current stream: the legacy default stream
    phi = torch.empty(n, dtype=torch.float32, device="cuda")
    force = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    for _ in range(2):  # capture + launch, replay
        _, _, e = plan.compute_batched_graph(counts, tp, tq, phi, force, energies=True)
        assert np.array_equal(phi.cpu().numpy(), rphi) and np.array_equal(force.cpu().numpy(), rforce)
        assert np.array_equal(e, re)
    plan.close()


@pytest.mark.parametrize("boundary,cutoff", [("periodic", 1), ("periodic", 2), ("open", 1)])
def test_split_evaluation_matches_plain_sequence(pk, boundary, cutoff):
    """near_field = NEAR_CELL_ITEMS_SPLIT: the far field runs on the plan's second stream
    beside the near field (PMMM_INFO_SPLIT = 1), plain and graph-launched, and
    gives the results of the one-stream sequence (stage timing on) bit for bit,
    energies included; the batched form too."""
    import torch
    bc = pk.PERIODIC if boundary == "periodic" else pk.OPEN
    cfg = pk.Config(mesh=(8, 8, 8), p=4, boundary=bc, precision=pk.FP32, cutoff=cutoff,
                    near_field=pk.NEAR_CELL_ITEMS_SPLIT)
    n = 32 * 8 ** 3  # 32 per cell: cell items, not the per-target kernel
    pos, q = synth.uniform_pm1(n, synth.seed(7, 10 + cutoff))
    tp = torch.tensor(pos.astype(np.float32), device="cuda")
    tq = torch.tensor(q.astype(np.float32), device="cuda")
    ref = pk.Plan(cfg)
    ref.set_timing(True)
    rphi, rforce, re = ref.compute(tp, tq, energy=True)
    assert ref.info(pk.INFO_SPLIT) == 0
    rphi, rforce = rphi.cpu().numpy(), rforce.cpu().numpy()
    counts = np.array([n // 2, 0, n - n // 2])
    bphi, bforce, be = ref.compute_batched(counts, tp, tq, energies=True)
    assert ref.info(pk.INFO_SPLIT) == 0
    bphi, bforce = bphi.cpu().numpy(), bforce.cpu().numpy()
    ref.close()

    plan = pk.Plan(cfg)
    phi = torch.empty(n, dtype=torch.float32, device="cuda")
    force = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    for k in range(3):  # plain, capture + launch, replay
        _, _, e = plan.compute(tp, tq, phi=phi, force=force, energy=True)
        assert plan.info(pk.INFO_SPLIT) == 1
        assert np.array_equal(phi.cpu().numpy(), rphi) and np.array_equal(force.cpu().numpy(), rforce), f"call {k}"
        assert e == re, f"call {k}"
    sphi, sforce, se = plan.compute_batched(counts, tp, tq, energies=True)
    assert plan.info(pk.INFO_SPLIT) == 1
    assert np.array_equal(sphi.cpu().numpy(), bphi) and np.array_equal(sforce.cpu().numpy(), bforce)
    assert np.array_equal(se, be)
    plan.close()
