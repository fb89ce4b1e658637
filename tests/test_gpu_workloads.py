"""The large-slice 53-qubit workload and the batch of 256 uneven circuits.

53 qubits has no state-vector oracle (2^53 amplitudes).  Slice 0 is checked
against the FP64 tensor-network oracle (oracle/tn.py, values stored by
tests/golden/make_golden.py grid53), in the configuration the benchmark
times; the other slices by invariants that hold at any size: the sum of
single-slice calls equals the range call (bit-identical for looped slices),
a plan that runs the slices batched gives the same sum, and the complex64
and FP16 paths agree on the same slices.

The uneven batch is checked circuit by circuit against the FP64 state vector
(live for the smaller circuits, stored oracle values for the others when
tests/golden/make_golden.py has written them)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
import rqcgen  # noqa: E402
import paper_2407_00769_gb300 as tn  # noqa: E402

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden", "batch")
GOLD53 = os.path.join(os.path.dirname(__file__), "golden")


def _grid53(dtype, batch=0):
    c, q = rqcgen.grid_53q()
    return tn.Plan(c, q, dtype=dtype, n_slice_edges=-1, max_log2_elems=30, trials=1,
                   slice_batch_log2=batch)


def test_grid53_slice_invariants():
    p16 = _grid53(tn.F16)
    info = p16.info()
    assert info["max_log2_elems"] <= 30 and info["n_open"] == 12
    whole = p16.contract(0, 4).cpu().numpy()
    acc = p16.contract(0, 1)
    for s in range(1, 4):
        p16.contract(s, 1, out=acc, accumulate=True)
    assert np.array_equal(acc.cpu().numpy(), whole)
    one16 = [p16.contract(s, 1).cpu().numpy() for s in range(2)]
    del p16
    torch.cuda.empty_cache()
    # batched slices: same sum, rounded differently (shared scale per pass)
    pb = _grid53(tn.F16, batch=2)
    assert oracle.rel_l2(pb.contract(0, 4).cpu().numpy(), whole) <= 5e-3
    del pb
    torch.cuda.empty_cache()
    # complex64 path on the same two slices
    p64 = _grid53(tn.C64)
    for s in range(2):
        c64 = p64.contract(s, 1).cpu().numpy()
        assert np.linalg.norm(c64) > 0
        assert oracle.rel_l2(one16[s], c64) <= 5e-3
        assert oracle.fidelity(c64, one16[s]) >= 0.999
    del p64
    torch.cuda.empty_cache()


def _read_amps(path):
    vals = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        _, a, b = line.split()
        vals.append(complex(float(a), float(b)))
    return np.array(vals)


def _read_plan(path):
    edges, leaves, steps = [], [], []
    for line in open(path):
        w = line.split()
        if not w or w[0].startswith("#"):
            continue
        {"edge": edges, "leaf": leaves, "step": steps}[w[0]].append((int(w[1]), int(w[2])))
    return edges, leaves, steps


@pytest.mark.parametrize("dtype,batch,tol", [(tn.C64, 0, 1e-5), (tn.F16, 3, 5e-3), (tn.BF16, 3, 2e-2)])
def test_grid53_slice0_against_network_oracle(dtype, batch, tol):
    want = _read_amps(os.path.join(GOLD53, "grid53_slice0.txt"))
    edges, _, steps = _read_plan(os.path.join(GOLD53, "grid53_plan.txt"))
    p = _grid53(dtype, batch=batch)
    # the stored values are for these sliced wires; the path only ordered
    # the oracle's work
    assert p.sliced_edges() == edges
    assert [tuple(sorted((s["a"], s["b"]))) for s in p.steps()] == [tuple(sorted(x)) for x in steps]
    got = p.contract(0, 1).cpu().numpy()
    del p
    torch.cuda.empty_cache()
    rel = oracle.rel_l2(got, want)
    print(f"53-qubit slice 0, {tn.DTYPE_NAMES[dtype]}: rel-L2 {rel:.2e} vs FP64 network oracle")
    assert rel <= tol
    assert oracle.fidelity(want, got) >= 0.999


def _golden(i):
    path = os.path.join(GOLD, f"circuit{i:03d}.txt")
    if not os.path.exists(path):
        return None
    vals = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        _, a, b = line.split()
        vals.append(complex(float(a), float(b)))
    return np.array(vals)


def test_uneven_batch_against_state_vector():
    # all 256 circuits as the benchmark runs them (plans within a 1 GiB
    # workspace, one graph over 16 streams): stored FP64 state-vector values,
    # or the live oracle for the circuits of <= 22 qubits when none is stored
    items = rqcgen.uneven_batch()
    idx, want = [], []
    for i in range(len(items)):
        c, q = items[i]
        w = _golden(i)
        if w is None and c.n_qubits <= 22:
            w = oracle.amplitudes(c, q)
        if w is not None:
            idx.append(i)
            want.append(w)
    assert len(idx) >= 64
    plans = [tn.plan_within_budget(*items[i], dtype=tn.F16) for i in idx]
    outs = [torch.zeros(64, dtype=torch.complex128, device="cuda") for _ in idx]
    b = tn.Batch(plans, outs, n_streams=16)
    b.run(stream=torch.cuda.Stream(), report=True)
    errs = []
    for o, w in zip(outs, want):
        got = o.cpu().numpy()
        errs.append(oracle.rel_l2(got, w))
        assert oracle.fidelity(w, got) >= 0.999
    print(f"uneven batch: {len(idx)} circuits, max rel-L2 {max(errs):.2e}, median {np.median(errs):.2e}")
    assert max(errs) <= 5e-3


def test_grid53_full_job_porter_thomas():
    # every slice of the 53-qubit circuit on an annealed path (512 slices at
    # cap 2^30): the 4096 probabilities of a deep random circuit follow the
    # Porter-Thomas law, 2^n p ~ Exp(1): mean 1 (+-0.05 at 3 sigma for 4096
    # values) and second moment 2 -- a property of the whole sum of slices
    c, q = rqcgen.grid_53q()
    p = tn.Plan(c, q, dtype=tn.F16, n_slice_edges=-1, max_log2_elems=30, trials=4, slice_batch_log2=3,
                anneal_iters=200000)
    amps = p.contract().cpu().numpy()
    del p
    torch.cuda.empty_cache()
    x = (2.0 ** 53) * np.abs(amps) ** 2
    print(f"53-qubit full job: mean 2^n p = {x.mean():.4f}, second moment {np.mean(x ** 2):.4f}")
    assert 0.93 <= x.mean() <= 1.07
    assert 1.6 <= np.mean(x ** 2) <= 2.4
    # recomputation (3 output legs split into 8 passes, 32 slices in all) on
    # its own path and slicing gives the same 4096 amplitudes: two FP16
    # computations, each within ~1e-3 of the exact values
    p = tn.Plan(c, q, dtype=tn.F16, n_slice_edges=-1, max_log2_elems=30, trials=4, slice_batch_log2=3,
                anneal_iters=200000, recompute_log2=3)
    assert p.info()["n_recompute_edges"] == 3
    amps_r = p.contract().cpu().numpy()
    del p
    torch.cuda.empty_cache()
    e = oracle.rel_l2(amps_r, amps)
    print(f"53-qubit full job with recomputation: rel-L2 {e:.2e} against the unsplit job")
    assert e <= 5e-3
