"""Pins of the sparse-state oracle (oracle/sparse.py, Sec. 3.4.2): the
paper's index example, the padded 2-D-index scheme against the direct
definition, and the direct definition against explicit sums."""
import numpy as np
import pytest

from oracle import sparse as gather


def test_paper_index_example():
    # Index_A = [0, 0, 1, 1, 1, 3, 4]: the value 1 repeats three times, so
    # the padded index has m_r = 3 columns (the paper's own example)
    ia = [0, 0, 1, 1, 1, 3, 4]
    ib = [5, 6, 7, 8, 9, 10, 11]
    P, where, m_r = gather.padded_index(ia, ib, m_a=5)
    assert m_r == 3
    assert P.tolist() == [[5, 6, -1], [7, 8, 9], [-1, -1, -1], [10, -1, -1], [11, -1, -1]]
    assert where.tolist() == [[0, 1, -1], [2, 3, 4], [-1, -1, -1], [5, -1, -1], [6, -1, -1]]
    with pytest.raises(ValueError):
        gather.padded_index([1, 0], [0, 0], m_a=2)


def _case(rng, m_a, m_b, m_n, M, K, N, sorted_a=True):
    A = rng.standard_normal((m_a, M, K)) + 1j * rng.standard_normal((m_a, M, K))
    B = rng.standard_normal((m_b, K, N)) + 1j * rng.standard_normal((m_b, K, N))
    ia = rng.integers(0, m_a, size=m_n)
    if sorted_a:
        ia = np.sort(ia)
    ib = rng.integers(0, m_b, size=m_n)
    return A, B, ia, ib


def test_direct_equals_explicit_sums():
    rng = np.random.default_rng(1)
    A, B, ia, ib = _case(rng, 3, 4, 6, 2, 4, 2, sorted_a=False)
    C = gather.direct(A, B, ia, ib)
    for n in range(6):
        for m in range(2):
            for j in range(2):
                s = 0j
                for k in range(4):
                    s += A[ia[n], m, k] * B[ib[n], k, j]
                assert abs(C[n, m, j] - s) <= 1e-13


@pytest.mark.parametrize("m_a,m_b,m_n", [(5, 3, 7), (8, 8, 40), (2, 9, 2), (16, 4, 16)])
def test_padded_scheme_equals_direct(m_a, m_b, m_n):
    rng = np.random.default_rng(m_a * 100 + m_n)
    A, B, ia, ib = _case(rng, m_a, m_b, m_n, 4, 8, 4)
    assert np.max(np.abs(gather.padded(A, B, ia, ib) - gather.direct(A, B, ia, ib))) <= 1e-12
