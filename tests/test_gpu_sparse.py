"""Sparse-state contraction of many tensor pairs (Sec. 3.4.2) on the tensor
cores, both index schemes, against the FP64 oracle (oracle/sparse.py) on
the same complex-half operands."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
from oracle import sparse  # noqa: E402
import paper_2407_00769_gb300 as tn  # noqa: E402

pytestmark = pytest.mark.gpu


def _operands(rng, m_a, m_b, M, K, N):
    a = (rng.standard_normal((m_a, M, K, 2))).astype(np.float16)
    b = (rng.standard_normal((m_b, K, N, 2)) / np.sqrt(K)).astype(np.float16)
    ac = a[..., 0].astype(np.float64) + 1j * a[..., 1].astype(np.float64)
    bc = b[..., 0].astype(np.float64) + 1j * b[..., 1].astype(np.float64)
    return torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), ac, bc


def _check(got, want, ac, bc, ia, ib):
    g = got.float().cpu().numpy().astype(np.float64)
    g = g[..., 0] + 1j * g[..., 1]
    mag = np.stack([np.abs(ac[i]) @ np.abs(bc[j]) for i, j in zip(ia, ib)])
    tol = 2 * 2.0 ** -11 * np.abs(want) + 1e-6 * mag + 1e-30
    assert np.all(np.abs(g - want) <= tol), float(np.max(np.abs(g - want) / (np.abs(want) + 1e-9)))


@pytest.mark.parametrize("scheme", [tn.GATHER_DIRECT, tn.GATHER_PADDED])
@pytest.mark.parametrize("m_a,m_b,m_n,M,K,N", [(37, 11, 100, 256, 64, 8), (5, 3, 7, 128, 8, 2),
                                                (1, 1, 1, 128, 16, 16), (64, 9, 300, 128, 1024, 4),
                                                (8, 200, 40, 256, 32, 128)])
def test_gather_contraction_against_oracle(scheme, m_a, m_b, m_n, M, K, N):
    rng = np.random.default_rng(m_a * 7 + m_n)
    A, B, ac, bc = _operands(rng, m_a, m_b, M, K, N)
    ia = np.sort(rng.integers(0, m_a, size=m_n))
    ia[-1] = m_a - 1                       # the last chunk is used
    ib = rng.integers(0, m_b, size=m_n)
    C = torch.full((m_n, M, N, 2), float("nan"), dtype=torch.float16, device="cuda")
    mx = torch.zeros(1, dtype=torch.float32, device="cuda")
    m_r = tn.gemm_gather(tn.F16, A, B, C, ia, ib, scheme=scheme, out_max=mx)
    want = sparse.direct(ac, bc, ia, ib)
    _check(C, want, ac, bc, ia, ib)
    if scheme == tn.GATHER_PADDED:
        assert m_r == sparse.padded_index(ia, ib, m_a)[2]
    g = C.float().cpu().numpy()
    assert abs(mx.item() - np.abs(g).max()) <= 1e-6 * np.abs(g).max()


def test_gather_unsorted_direct_and_padded_rejects_unsorted():
    rng = np.random.default_rng(3)
    A, B, ac, bc = _operands(rng, 6, 4, 128, 32, 8)
    ia = rng.integers(0, 6, size=20)
    ib = rng.integers(0, 4, size=20)
    C = torch.zeros(20, 128, 8, 2, dtype=torch.float16, device="cuda")
    tn.gemm_gather(tn.F16, A, B, C, ia, ib, scheme=tn.GATHER_DIRECT)
    _check(C, sparse.direct(ac, bc, ia, ib), ac, bc, ia, ib)
    if np.any(np.diff(ia) < 0):
        with pytest.raises(tn.TnError):
            tn.gemm_gather(tn.F16, A, B, C, ia, ib, scheme=tn.GATHER_PADDED)


def test_gather_bf16():
    rng = np.random.default_rng(5)
    m_a, m_b, m_n, M, K, N = 9, 4, 30, 128, 64, 16
    a = rng.standard_normal((m_a, M, K, 2))
    b = rng.standard_normal((m_b, K, N, 2)) / np.sqrt(K)
    A = torch.from_numpy(a).float().cuda().to(torch.bfloat16)
    B = torch.from_numpy(b).float().cuda().to(torch.bfloat16)
    ar = A.float().cpu().numpy().astype(np.float64)
    br = B.float().cpu().numpy().astype(np.float64)
    ac, bc = ar[..., 0] + 1j * ar[..., 1], br[..., 0] + 1j * br[..., 1]
    ia = np.sort(rng.integers(0, m_a, size=m_n))
    ib = rng.integers(0, m_b, size=m_n)
    C = torch.zeros(m_n, M, N, 2, dtype=torch.bfloat16, device="cuda")
    tn.gemm_gather(tn.BF16, A, B, C, ia, ib, scheme=tn.GATHER_PADDED)
    g = C.float().cpu().numpy().astype(np.float64)
    g = g[..., 0] + 1j * g[..., 1]
    want = sparse.padded(ac, bc, ia, ib)
    assert np.linalg.norm(g - want) / np.linalg.norm(want) < 2 * 2.0 ** -8
