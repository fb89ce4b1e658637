"""Recomputation (Sec. 3.4.1): open output legs split into sequential
passes, each filling its part of the amplitude vector (concatenation, not a
sum).  Checked against the FP64 state vector and the stored FP64 amplitudes
of the 30-qubit workload; partial slice ranges fill exactly their parts."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
import rqcgen  # noqa: E402
import paper_2407_00769_gb300 as tn  # noqa: E402

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold30():
    rows = [l.split() for l in open(os.path.join(GOLD, "grid5x6_14c_amps.txt")) if not l.startswith("#")]
    return np.array([complex(float(r[1]), float(r[2])) for r in rows])


@pytest.mark.parametrize("dtype,r,slices,batch", [(tn.C64, 1, 0, 0), (tn.C64, 2, 2, 1), (tn.F16, 3, 3, 2),
                                                  (tn.F16, 1, 2, 2)])
def test_recompute_matches_state_vector(dtype, r, slices, batch):
    c, q = rqcgen.small_grid(3, 4, 8, seed=3, n_open=6)
    p = tn.Plan(c, q, dtype=dtype, n_slice_edges=slices, slice_batch_log2=batch, recompute_log2=r)
    info = p.info()
    assert info["n_recompute_edges"] == r and info["n_slices"] == 1 << (slices + r)
    split_qubits = [qq for qq, _ in p.sliced_edges()[-r:]]
    assert set(split_qubits) <= set(q.open_qubits)
    got = p.contract().cpu().numpy()
    want = oracle.amplitudes(c, q)
    assert oracle.rel_l2(got, want) <= (1e-5 if dtype == tn.C64 else 5e-3)


def test_recompute_parts_are_disjoint():
    # the slices of one part are contiguous: the first half of the slice
    # range fills exactly the amplitudes whose split bit is 0
    c, q = rqcgen.small_grid(3, 4, 8, seed=3, n_open=6)
    p = tn.Plan(c, q, dtype=tn.C64, n_slice_edges=2, recompute_log2=1)
    n = p.info()["n_slices"]
    full = p.contract().cpu().numpy()
    first = p.contract(0, n // 2).cpu().numpy()
    qq = p.sliced_edges()[-1][0]
    t = list(q.open_qubits).index(qq)
    part0 = ((np.arange(full.size) >> t) & 1) == 0
    assert np.all(first[~part0] == 0)
    assert np.allclose(first[part0], full[part0], rtol=0, atol=1e-12)
    both = p.contract(0, n // 2)
    p.contract(n // 2, n - n // 2, out=both, accumulate=True)
    assert np.allclose(both.cpu().numpy(), full, rtol=0, atol=1e-12)


def test_recompute_30_qubits_full_size():
    gold = _gold30()
    c, q = rqcgen.grid_30q()
    p = tn.Plan(c, q, dtype=tn.F16, n_slice_edges=8, trials=4, slice_batch_log2=8, recompute_log2=1)
    amps = p.contract()
    m = tn.metrics(amps, torch.from_numpy(gold).cuda(), n_qubits=30)
    print(f"30-qubit, 1 split leg: rel-L2 {m['rel_l2']:.2e}, {p.info()['n_slices']} slices")
    assert m["rel_l2"] <= 5e-3 and m["fidelity"] >= 0.999
