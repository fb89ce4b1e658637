"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the GPU library
(``paper_2407_00769_gb300``) and never imports it; both take their inputs from
``rqcgen``.  Every function is plain and slow on purpose.

Contents
  * state_vector / amplitudes: the state-vector method (paper Sec. 2), FP64,
    with optional wire projectors that define one slice of a sliced network
    (paper Sec. 3.1: sub-networks from broken edges).      -> oracle/sv.c
  * bruteforce_state: product of full 2^n x 2^n gate matrices (n <= 8).
  * complex_as_real_einsum: the paper's complex-half einsum extension
    (Sec. 3.3, Eq. 5-6), FP64, pinned by the paper's worked example.
  * rel_l2, fidelity (Eq. 8), linear_xeb, topk (post-selection, Sec. 1/2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Iterable, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle/sv.c with gcc (OpenMP, -O2, plain C11)."""
    src = os.path.join(_HERE, "sv.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", src,
           "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        f64p = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.oracle_sv_run.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, f64p, f64p,
                                      ctypes.c_int, i32p, i32p, i32p, f64p]
        lib.oracle_sv_run.restype = ctypes.c_int
        lib.oracle_gather.argtypes = [ctypes.c_int, f64p, ctypes.c_int, i32p, u8p, f64p]
        lib.oracle_gather.restype = None
        lib.oracle_bruteforce.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, f64p, f64p, f64p]
        lib.oracle_bruteforce.restype = ctypes.c_int
        lib.oracle_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def threads() -> int:
    return int(_load().oracle_threads())


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _gate_arrays(circuit):
    q0 = np.ascontiguousarray(circuit.q0, dtype=np.int32)
    q1 = np.ascontiguousarray(circuit.q1, dtype=np.int32)
    mats = np.asarray(circuit.mats, dtype=np.complex128).reshape(-1, 16)
    return q0, q1, np.ascontiguousarray(mats.real), np.ascontiguousarray(mats.imag)


def state_vector(circuit, projectors: Optional[Sequence] = None) -> np.ndarray:
    """|psi> = U|0^n> in FP64 (2^n complex128), qubit q = bit q of the index.

    ``projectors``: iterable of (qubit, after_gate, value); |value><value| is
    applied to ``qubit`` right after gate ``after_gate`` (-1: before gate 0).
    """
    lib = _load()
    n = int(circuit.n_qubits)
    q0, q1, re, im = _gate_arrays(circuit)
    pr = list(projectors or [])
    pq = np.array([p[0] for p in pr] or [0], dtype=np.int32)
    pa = np.array([p[1] for p in pr] or [0], dtype=np.int32)
    pv = np.array([p[2] for p in pr] or [0], dtype=np.int32)
    psi = np.empty(1 << n, dtype=np.complex128)
    rc = lib.oracle_sv_run(n, q0.shape[0], _ptr(q0, ctypes.c_int32), _ptr(q1, ctypes.c_int32),
                           _ptr(re, ctypes.c_double), _ptr(im, ctypes.c_double),
                           len(pr), _ptr(pq, ctypes.c_int32), _ptr(pa, ctypes.c_int32),
                           _ptr(pv, ctypes.c_int32), _ptr(psi.view(np.float64), ctypes.c_double))
    if rc != 0:
        raise ValueError(f"oracle_sv_run rejected the circuit (rc={rc})")
    return psi


def gather(circuit, query, psi: np.ndarray) -> np.ndarray:
    """amp[j] = psi[x(j)]: bit t of j on open_qubits[t], fixed bits elsewhere."""
    lib = _load()
    oq = np.ascontiguousarray(query.open_qubits, dtype=np.int32)
    fb = np.ascontiguousarray(query.fixed_bits, dtype=np.uint8)
    out = np.empty(1 << int(oq.shape[0]), dtype=np.complex128)
    lib.oracle_gather(int(circuit.n_qubits), _ptr(psi.view(np.float64), ctypes.c_double),
                      int(oq.shape[0]), _ptr(oq, ctypes.c_int32), _ptr(fb, ctypes.c_uint8),
                      _ptr(out.view(np.float64), ctypes.c_double))
    return out


def amplitudes(circuit, query, projectors: Optional[Sequence] = None) -> np.ndarray:
    """The queried amplitudes <x|U|0^n> (optionally of one slice)."""
    return gather(circuit, query, state_vector(circuit, projectors))


def slice_projectors(sliced_edges: Sequence, slice_id: int):
    """Projectors of one slice.  ``sliced_edges[j] = (qubit, after_gate)``;
    bit j of ``slice_id`` (LSB first) is the wire's fixed value."""
    return [(int(q), int(g), (int(slice_id) >> j) & 1) for j, (q, g) in enumerate(sliced_edges)]


def sliced_amplitudes(circuit, query, sliced_edges, slice_ids: Iterable[int]) -> np.ndarray:
    """Sum over ``slice_ids`` (ascending order) of each slice's amplitudes."""
    acc = None
    for s in sorted(int(x) for x in slice_ids):
        a = amplitudes(circuit, query, slice_projectors(sliced_edges, s))
        acc = a if acc is None else acc + a
    return acc


def bruteforce_state(circuit) -> np.ndarray:
    """Column 0 of the full unitary product (n <= 8 recommended)."""
    lib = _load()
    n = int(circuit.n_qubits)
    q0, q1, re, im = _gate_arrays(circuit)
    out = np.empty(1 << n, dtype=np.complex128)
    rc = lib.oracle_bruteforce(n, q0.shape[0], _ptr(q0, ctypes.c_int32), _ptr(q1, ctypes.c_int32),
                               _ptr(re, ctypes.c_double), _ptr(im, ctypes.c_double),
                               _ptr(out.view(np.float64), ctypes.c_double))
    if rc != 0:
        raise ValueError(f"oracle_bruteforce failed (rc={rc})")
    return out


# --------------------------------------------------------------------------
# Complex-half einsum extension (paper Sec. 3.3, Eq. 5-6)
# --------------------------------------------------------------------------

def pad_b(b: np.ndarray) -> np.ndarray:
    """B (complex, any shape S) -> B' (real, shape (2,) + S + (2,)).

    B' carries a new leading output mode (the result's real/imag selector)
    and a trailing mode shared with A's real/imag mode:
      B'[0, ..., 0] = Re B,  B'[0, ..., 1] = -Im B,
      B'[1, ..., 0] = Im B,  B'[1, ..., 1] =  Re B.
    """
    b = np.asarray(b)
    out = np.empty((2,) + b.shape + (2,), dtype=np.float64)
    out[0, ..., 0] = b.real
    out[0, ..., 1] = -b.imag
    out[1, ..., 0] = b.imag
    out[1, ..., 1] = b.real
    return out


def complex_as_real_einsum(eq: str, a_real: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Evaluate the complex einsum ``eq`` ("A,B->C", single-letter modes) the
    paper's way: A is given as real with its real/imag mode last, B is padded
    to B' (``pad_b``), and one real einsum runs over the modified equation
    "A r, o B r -> C o" (Eq. 6).  Returns C real with its real/imag mode last.
    """
    lhs, out = eq.replace(" ", "").split("->")
    ea, eb = lhs.split(",")
    used = set(ea + eb + out)
    spare = [c for c in "zyxwvutsrqponmlkjihgfedcba" if c not in used]
    r, o = spare[0], spare[1]
    mod = f"{ea}{r},{o}{eb}{r}->{out}{o}"
    return np.einsum(mod, np.asarray(a_real, dtype=np.float64), pad_b(b))


# --------------------------------------------------------------------------
# Metrics (FP64)
# --------------------------------------------------------------------------

def rel_l2(result: np.ndarray, reference: np.ndarray) -> float:
    """||r - b||_2 / ||b||_2 over the complex vector."""
    r = np.asarray(result, dtype=np.complex128).ravel()
    b = np.asarray(reference, dtype=np.complex128).ravel()
    return float(np.linalg.norm(r - b) / np.linalg.norm(b))


def fidelity(reference: np.ndarray, result: np.ndarray) -> float:
    """Eq. 8 read for complex vectors: |<b, r>|^2 / (||b||^2 ||r||^2) with the
    conjugate-linear inner product <b, r> = sum conj(b) r."""
    b = np.asarray(reference, dtype=np.complex128).ravel()
    r = np.asarray(result, dtype=np.complex128).ravel()
    ip = np.vdot(b, r)
    return float(abs(ip) ** 2 / (np.vdot(b, b).real * np.vdot(r, r).real))


def linear_xeb(sample_probs: np.ndarray, n_qubits: int) -> float:
    """Linear cross-entropy benchmark: 2^n * mean ideal probability - 1."""
    p = np.asarray(sample_probs, dtype=np.float64)
    return float((2.0 ** n_qubits) * p.mean() - 1.0)


def topk(amps: np.ndarray, k: int):
    """Indices and probabilities |amp|^2 = re*re + im*im (each product and the
    sum rounded once, FP64) of the k largest; ties go to the lower index.
    Plain: a stable sort on (-p, index)."""
    a = np.asarray(amps, dtype=np.complex128)
    p = a.real * a.real + a.imag * a.imag
    idx = np.lexsort((np.arange(p.shape[0]), -p))[:k]
    return idx.astype(np.int64), p[idx]
