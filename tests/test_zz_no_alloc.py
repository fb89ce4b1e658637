"""tn_sample_noalloc: post-selection for callers that cannot allocate device
memory (a plug-in inside a host application that owns all device memory, or
a latency-critical thread that must not enter the CUDA allocator).  Its
results must equal tn_sample's, call after call, although every call shares
one fixed scratch array that keeps the previous call's contents.

Kept in a file of its own that pytest collects last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2407_00769_gb300 as tn  # noqa: E402

pytestmark = pytest.mark.gpu


def _amps(seed, n_open):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(1 << n_open) + 1j * rng.standard_normal(1 << n_open)
    a[[3, 17, 40]] = a[5]   # equal probabilities: ties go to the lower index
    return torch.from_numpy(a).cuda()


def _call(name, amps, k):
    L = tn.lib()
    n_open = amps.numel().bit_length() - 1
    idx = np.full(k, -7, dtype=np.int64)
    prob = np.full(k, -7.0)
    stream = torch.cuda.current_stream().cuda_stream
    rc = getattr(L, name)(amps.data_ptr(), n_open, k, idx.ctypes.data, prob.ctypes.data, stream)
    assert rc == tn.TN_OK, L.tn_last_error()
    return idx, prob


def test_noalloc_matches_tn_sample_on_consecutive_calls():
    # a large k, then a smaller k on other data: the second call must not
    # see anything left in the shared scratch by the first
    # (the first two cases take the multi-block selection, which uses the
    # rest of the fixed scratch; the others the one-block kernel)
    for seed, n_open, k in ((5, 20, 1000), (6, 16, 300), (1, 12, 1024), (2, 10, 37), (3, 6, 64)):
        amps = _amps(seed, n_open)
        got_idx, got_prob = _call("tn_sample_noalloc", amps, k)
        want_idx, want_prob = _call("tn_sample", amps, k)
        assert np.array_equal(got_idx, want_idx)
        assert np.array_equal(got_prob, want_prob)


def test_noalloc_rejects_k_beyond_its_scratch():
    amps = _amps(4, 12)
    L = tn.lib()
    idx = np.zeros(2048, dtype=np.int64)
    prob = np.zeros(2048)
    rc = L.tn_sample_noalloc(amps.data_ptr(), 12, 1025, idx.ctypes.data, prob.ctypes.data,
                             torch.cuda.current_stream().cuda_stream)
    assert rc == tn.TN_EINVAL
    assert b"exceeds its fixed scratch" in L.tn_last_error()
