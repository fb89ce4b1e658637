"""Top-k post-selection (Sec. 1 and Sec. 2, post-processing) at sizes where
the multi-block selection runs (k * 2^n_open > 2^22): radix select over the
bits of |amp|^2, collection of the k kept entries, bitonic sort.  Results
must equal the oracle's stable sort on (-p, index) exactly -- indices and
probabilities -- including ties at the threshold and k beyond the
shared-memory sort."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
import paper_2407_00769_gb300 as tn  # noqa: E402

pytestmark = pytest.mark.gpu


def _check(a, k):
    idx, prob = tn.sample(torch.from_numpy(a).cuda(), k)
    widx, wprob = oracle.topk(a, k)
    assert np.array_equal(idx, widx)
    assert np.array_equal(prob, wprob)


def test_topk_24_open_qubits_k1024():
    rng = np.random.default_rng(24)
    n = 1 << 24
    a = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * 2.0 ** -12
    _check(a, 1024)
    _check(a, 1)


@pytest.mark.parametrize("k", [1, 777, 2048, 2049, 5000])
def test_topk_heavy_ties(k):
    # few distinct probabilities: the threshold value is shared by many
    # entries, of which exactly the lowest indices must be kept
    rng = np.random.default_rng(k)
    n = 1 << 20
    vals = np.array([0, 0.5, 1, 1j, -1, 0.5j, 0.25 + 0.25j], dtype=np.complex128)
    a = vals[rng.integers(0, len(vals), size=n)]
    _check(a, k)


def test_topk_every_entry_and_signed_zeros():
    # k = n (global bitonic sort of every entry); -0.0 and +0.0 give the same p
    rng = np.random.default_rng(3)
    n = 1 << 14
    a = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    a[::7] = complex(-0.0, 0.0)
    a[1::7] = complex(0.0, -0.0)
    _check(a, n)
