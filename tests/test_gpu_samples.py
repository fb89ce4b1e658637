"""Amplitudes of arbitrary (uncorrelated) bitstrings: tn_plan_samples
carries the sample index as batch hyperedges through the contraction.
Checked against the FP64 state vector at those bitstrings, and at full size
against the stored amplitudes of the 30-qubit workload (bitstrings drawn
from its correlated subspace)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
import rqcgen  # noqa: E402
import paper_2407_00769_gb300 as tn  # noqa: E402

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
TOL = {tn.C64: 1e-5, tn.F16: 5e-3}


def _sv_at(c, samples):
    psi = oracle.state_vector(c)
    idx = (samples.astype(np.int64) << np.arange(samples.shape[1], dtype=np.int64)).sum(axis=1)
    return psi[idx]


@pytest.mark.parametrize("dtype", [tn.C64, tn.F16])
@pytest.mark.parametrize("n_samples,slices,batch", [(10, 2, 0), (64, 3, 2), (1, 0, 0), (1000, 2, 1), (257, 4, 4), (33, 3, 3)])
def test_sample_amplitudes_against_state_vector(dtype, n_samples, slices, batch):
    c, _ = rqcgen.small_grid(3, 4, 8, seed=3, n_open=4)
    rng = np.random.default_rng(n_samples + slices)
    samples = rng.integers(0, 2, size=(n_samples, c.n_qubits))
    p = tn.Plan.from_samples(c, samples, dtype=dtype, n_slice_edges=slices, slice_batch_log2=batch)
    got = p.contract().cpu().numpy()
    assert got.shape[0] == 1 << p.n_open and p.n_open == int(np.ceil(np.log2(max(n_samples, 1))))
    got = got[:n_samples]
    want = _sv_at(c, samples)
    assert oracle.rel_l2(got, want) <= TOL[dtype]
    assert oracle.fidelity(want, got) >= 0.999


def test_sample_amplitudes_30_qubits_full_size():
    path = os.path.join(GOLD, "grid5x6_14c_amps.txt")
    gold = np.array([complex(float(l.split()[1]), float(l.split()[2])) for l in open(path)
                     if not l.startswith("#")])
    c, q = rqcgen.grid_30q()
    rng = np.random.default_rng(7)
    j = rng.choice(1024, size=64, replace=False)
    samples = np.zeros((64, 30), dtype=np.uint8)
    samples[:, :] = np.asarray(q.fixed_bits, dtype=np.uint8)[None, :]
    for t, qq in enumerate(q.open_qubits):
        samples[:, qq] = (j >> t) & 1
    p = tn.Plan.from_samples(c, samples, dtype=tn.F16, n_slice_edges=8, trials=4, slice_batch_log2=4)
    got = p.contract().cpu().numpy()[:64]
    e = oracle.rel_l2(got, gold[j])
    print(f"30-qubit, 64 bitstrings, FP16: rel-L2 {e:.2e}")
    assert e <= 5e-3


def test_sample_plan_rejects_bad_bits():
    c, _ = rqcgen.small_grid(2, 2, 4, seed=1, n_open=1)
    with pytest.raises(tn.TnError):
        tn.Plan.from_samples(c, np.full((3, 4), 2), dtype=tn.C64)
