"""Sparse-state contraction of many tensor pairs -- TEST INFRASTRUCTURE ONLY.

Sec. 3.4.2 ("Tensor contraction during sparse state"), in the paper's
notation: A[a, c, d, f] and B[b, e, f] hold m_a and m_b chunks (the
outermost ranks a and b), the other modes have dimension 2, and f is
contracted.  With index arrays Index_A, Index_B of m_n entries,

    C[n, c, d, e] = sum_f A[Index_A[n], c, d, f] B[Index_B[n], e, f]     (direct)

The second scheme avoids gathering A when Index_A repeats its entries (it
is sorted, e.g. [0, 0, 1, 1, 1, 3, 4]): Index_B becomes a 2-D index P of
shape m_a x m_r, m_r the largest number of repeats of one value in Index_A,
row i listing the B chunks paired with A chunk i and -1 in the unused
places; B_P[i, r] = B[P[i, r]] (zero where P is -1); C_P = A x B_P chunk by
chunk; C is read back out of C_P at the valid places, in the order of n.

Written with plain loops and ``np.matmul`` per chunk (FP64, complex).
A chunk is an M x K matrix (the modes c, d flattened, f last), a B chunk
K x N (e flattened; stored [f][e], i.e. as the right-hand factor).
"""
from __future__ import annotations

from typing import Tuple

import numpy as np


def direct(A: np.ndarray, B: np.ndarray, index_a, index_b) -> np.ndarray:
    """C[n] = A[index_a[n]] @ B[index_b[n]]."""
    A = np.asarray(A, dtype=np.complex128)
    B = np.asarray(B, dtype=np.complex128)
    out = np.empty((len(index_a), A.shape[1], B.shape[2]), dtype=np.complex128)
    for n, (ia, ib) in enumerate(zip(index_a, index_b)):
        out[n] = np.matmul(A[ia], B[ib])
    return out


def padded_index(index_a, index_b, m_a: int) -> Tuple[np.ndarray, np.ndarray, int]:
    """(P, where, m_r): P[i, r] = the B chunk of the r-th n with index_a[n] = i
    (-1 where unused), where[i, r] = that n (-1 where unused).  index_a must
    be non-decreasing."""
    index_a = list(index_a)
    if any(index_a[i] > index_a[i + 1] for i in range(len(index_a) - 1)):
        raise ValueError("index_a must be sorted")
    counts = np.zeros(m_a, dtype=np.int64)
    for ia in index_a:
        counts[ia] += 1
    m_r = int(counts.max()) if len(index_a) else 0
    P = -np.ones((m_a, m_r), dtype=np.int64)
    where = -np.ones((m_a, m_r), dtype=np.int64)
    fill = np.zeros(m_a, dtype=np.int64)
    for n, (ia, ib) in enumerate(zip(index_a, index_b)):
        P[ia, fill[ia]] = ib
        where[ia, fill[ia]] = n
        fill[ia] += 1
    return P, where, m_r


def padded(A: np.ndarray, B: np.ndarray, index_a, index_b) -> np.ndarray:
    """The second scheme: C_P[i] = A[i] x B_P[i] (B_P[i] = the m_r chunks of
    row i of P side by side, zeros for -1), then the valid places of C_P in
    the order of n."""
    A = np.asarray(A, dtype=np.complex128)
    B = np.asarray(B, dtype=np.complex128)
    m_a, M, K = A.shape
    N = B.shape[2]
    P, where, m_r = padded_index(index_a, index_b, m_a)
    CP = np.zeros((m_a, M, m_r * N), dtype=np.complex128)
    for i in range(m_a):
        BP = np.zeros((K, m_r * N), dtype=np.complex128)
        for r in range(m_r):
            if P[i, r] >= 0:
                BP[:, r * N:(r + 1) * N] = B[P[i, r]]
        CP[i] = np.matmul(A[i], BP)
    out = np.empty((len(index_a), M, N), dtype=np.complex128)
    for i in range(m_a):
        for r in range(m_r):
            n = where[i, r]
            if n >= 0:
                out[n] = CP[i][:, r * N:(r + 1) * N]
    return out
