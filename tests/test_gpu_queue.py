"""The persistent work-queue launch (tn_queue_*, tn_plan_set_queue): many
plans' whole contractions -- every slice pass, every step -- as one kernel
launch whose CTAs claim (op, tile) items in dependency order.

Parity: the queue runs the same device code as the stream of stand-alone
launches (shared bodies, the same tcgen05 pipeline), so its amplitudes must
equal tn_contract's BIT FOR BIT, and through that the FP64 oracle within the
path's tolerance (complex64 1e-5, FP16 5e-3).  The queue's bounded wait
is run to its timeout on purpose (an op that nothing lists) and the context
is then used again."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
import rqcgen  # noqa: E402
import paper_2407_00769_gb300 as tn  # noqa: E402

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
TOL = {tn.C64: 1e-5, tn.F16: 5e-3, tn.BF16: 2e-2}


def _bits(t):
    return t.cpu().numpy().view(np.uint64).copy()


def _stream_and_queue(make_plan, begin=0, count=None):
    p = make_plan()
    n_open = p.info()["n_open"]
    want = torch.zeros(1 << n_open, dtype=torch.complex128, device="cuda")
    p.contract(begin, count, out=want)
    q = make_plan()
    got = torch.zeros_like(want)
    qu = tn.Queue([q], [got], ranges=None if count is None else [(begin, count)])
    qu.run(report=True)
    torch.cuda.synchronize()
    return want, got, qu.info()


def test_queue_wait_runs_out_and_context_survives():
    s = torch.cuda.Stream()
    assert tn.selftest_queue_timeout(200, stream=s) == tn.TN_ETIMEOUT
    # the context is intact: a queued contraction right after
    c, q = rqcgen.grid_12q()
    p = tn.Plan(c, q, dtype=tn.F16, small_log2=6)
    out = torch.zeros(4096, dtype=torch.complex128, device="cuda")
    tn.Queue([p], [out]).run(report=True)
    assert oracle.rel_l2(out.cpu().numpy(), oracle.amplitudes(c, q)) <= 5e-3


@pytest.mark.parametrize("dtype,small,slices,batch", [
    (tn.C64, 0, 0, 0), (tn.F16, 6, 0, 0), (tn.F16, 6, 3, 0), (tn.F16, 6, 3, 2), (tn.BF16, 6, 2, 1),
    (tn.F16, 0, 2, 0), (tn.C64, 0, 3, 1)])
def test_queue_equals_stream_bit_for_bit(dtype, small, slices, batch):
    # 12-qubit grid, all 4096 amplitudes; small_log2 = 6 puts the tcgen05
    # steps (and B' builds) on this circuit, so every op kind is queued
    c, q = rqcgen.grid_12q()

    def mk():
        return tn.Plan(c, q, dtype=dtype, small_log2=small, n_slice_edges=slices, slice_batch_log2=batch)

    want, got, info = _stream_and_queue(mk)
    assert info["n_items"] >= info["n_ops"] > 10
    assert (_bits(got) == _bits(want)).all()
    e = oracle.rel_l2(got.cpu().numpy(), oracle.amplitudes(c, q))
    assert e <= TOL[dtype], e


def test_queue_partial_slice_range_bit_for_bit():
    # slices [3, 3 + 5) of 16, two slices per pass: a ragged first and last pass
    c, q = rqcgen.small_grid(4, 4, 10, seed=3, n_open=5)

    def mk():
        return tn.Plan(c, q, dtype=tn.F16, small_log2=4, n_slice_edges=4, slice_batch_log2=1)

    want, got, _ = _stream_and_queue(mk, begin=3, count=5)
    assert (_bits(got) == _bits(want)).all()
    edges = mk().sliced_edges()
    ref = oracle.sliced_amplitudes(c, q, edges, range(3, 8))
    assert oracle.rel_l2(got.cpu().numpy(), ref) <= 5e-3


def test_queue_recompute_and_samples_bit_for_bit():
    c, q = rqcgen.small_grid(4, 4, 10, seed=5, n_open=6)

    def mk():
        return tn.Plan(c, q, dtype=tn.F16, small_log2=4, n_slice_edges=2, recompute_log2=2)

    want, got, _ = _stream_and_queue(mk)
    assert (_bits(got) == _bits(want)).all()
    assert oracle.rel_l2(got.cpu().numpy(), oracle.amplitudes(c, q)) <= 5e-3
    # uncorrelated bitstrings (sparse-state gather steps)
    rng = np.random.default_rng(7)
    samples = rng.integers(0, 2, size=(37, c.n_qubits)).astype(np.uint8)

    def mks():
        return tn.Plan.from_samples(c, samples, dtype=tn.F16, small_log2=4, n_slice_edges=2)

    want, got, _ = _stream_and_queue(mks)
    assert (_bits(got) == _bits(want)).all()


def _golden(i):
    path = os.path.join(GOLD, "batch", f"circuit{i:03d}.txt")
    vals = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        _, a, b = line.split()
        vals.append(complex(float(a), float(b)))
    return np.array(vals)


def test_queue_uneven_circuits_one_launch():
    # 48 circuits of the uneven batch (every fifth, 16-28 qubits) in one
    # launch: equal to their stand-alone contractions bit for bit, and to the
    # stored FP64 state-vector amplitudes within the FP16 budget
    items = rqcgen.uneven_batch()
    idx = list(range(0, 240, 5))
    plans = [tn.plan_within_budget(*items[i], dtype=tn.F16) for i in idx]
    outs = [torch.zeros(64, dtype=torch.complex128, device="cuda") for _ in idx]
    qu = tn.Queue(plans, outs)
    rep = qu.run(stream=torch.cuda.Stream(), report=True)
    assert rep["kernels"] == 1
    info = qu.info()
    assert info["n_plans"] == len(idx)
    errs = []
    for i, p, o in zip(idx, plans, outs):
        ref = torch.zeros_like(o)
        p.contract(out=ref)
        assert (_bits(o) == _bits(ref)).all(), i
        w = _golden(i)
        errs.append(oracle.rel_l2(o.cpu().numpy(), w))
        assert oracle.fidelity(w, o.cpu().numpy()) >= 0.999
    print(f"queue: {len(idx)} circuits, {info['n_items']} items, {info['n_ops']} ops, "
          f"max rel-L2 {max(errs):.2e}, {rep['ms']:.1f} ms")
    assert max(errs) <= 5e-3


def test_queue_rerun_is_deterministic():
    c, q = rqcgen.grid_12q()
    p = tn.Plan(c, q, dtype=tn.F16, small_log2=6, n_slice_edges=3)
    out = torch.zeros(4096, dtype=torch.complex128, device="cuda")
    qu = tn.Queue([p], [out])
    qu.run()
    first = _bits(out)
    for _ in range(3):
        qu.run()
        assert (_bits(out) == first).all()


def test_plan_set_queue_full_size_30_qubits():
    # the benchmark's workload (30 qubits, 256 slices in one pass, FP16,
    # tuned tiles) as one queued launch: equal to the stream path bit for
    # bit and within 5e-3 of the stored FP64 amplitudes
    c, q = rqcgen.grid_30q()
    p = tn.Plan(c, q, dtype=tn.F16, n_slice_edges=8, trials=4, slice_batch_log2=8, tile_policy=tn.TILE_EXHAUSTIVE)
    want = p.contract()
    p.set_queue(True)
    got = p.contract()
    torch.cuda.synchronize()
    assert (_bits(got) == _bits(want)).all()
    gold = []
    for line in open(os.path.join(GOLD, "grid5x6_14c_amps.txt")):
        if line.startswith("#") or not line.strip():
            continue
        _, a, b = line.split()
        gold.append(complex(float(a), float(b)))
    assert oracle.rel_l2(got.cpu().numpy(), np.array(gold)) <= 5e-3


def test_queue_annealed_circuits_with_split_k_steps():
    # annealed paths of uneven circuits carry tensor-core steps with few
    # output tiles, which the library splits along K (FP32 partials summed in
    # FP64 by a separate op); the queue runs those parts and reductions too
    items = rqcgen.uneven_batch()
    idx = [2, 7, 12, 22, 31, 40]
    plans = [tn.plan_within_budget(*items[i], dtype=tn.F16, anneal_iters=20000) for i in idx]
    outs = [torch.zeros(64, dtype=torch.complex128, device="cuda") for _ in idx]
    qu = tn.Queue(plans, outs)
    qu.profile(True)
    qu.run(report=True)
    prof = qu.profile_read()
    assert prof.get("splitk", {}).get("items", 0) > 0, prof
    for i, p, o in zip(idx, plans, outs):
        ref = torch.zeros_like(o)
        p.contract(out=ref)
        assert (_bits(o) == _bits(ref)).all(), i
        assert oracle.rel_l2(o.cpu().numpy(), _golden(i)) <= 5e-3
