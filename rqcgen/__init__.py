"""Seeded synthetic Sycamore-shaped random quantum circuits (inputs only).

This module is the one place that both the CPU oracle (``oracle/``) and the
GPU library (``paper_2407_00769_gb300``) take their inputs from.  It holds no
arithmetic of the contraction method: it only draws circuits and queries.

Circuit model (paper Sec. 2, "circuit structure"): m full cycles, each a layer
of single-qubit gates on every qubit followed by two-qubit gates on the qubit
pairs that the cycle's coupler pattern selects, then a half cycle of
single-qubit gates before all qubits are measured.  Gate set (same section):
sqrt(X), sqrt(Y), sqrt(W) and fSim(theta, phi).

Readings where the paper is silent:
  * 1q gate draw: one splitmix64 stream per circuit seeded with ``seed``;
    first layer uniform over {sqrt(X), sqrt(Y), sqrt(W)}: ``(u >> 11) % 3``;
    later layers uniform over the two gates that differ from the previous one
    on that qubit: ``(u >> 11) % 2`` indexes them in ascending gate order.
    Draws go layer by layer, qubit by qubit in ascending index.
  * fSim(theta=pi/2, phi=pi/6) on every pair.
  * Coupler pattern "ABCD" repeating on an R x C rectilinear grid, qubit
    (r, c) -> r*C + c (removed sites skipped, renumbered row-major):
    A = horizontal (r,c)-(r,c+1), c even; B = horizontal, c odd;
    C = vertical (r,c)-(r+1,c), r even; D = vertical, r odd.
    Cycle k uses pattern k mod 4.  Gates of a layer are listed row-major by
    their first site, horizontal partner before vertical.
  * Fixed (non-open) output bits: a splitmix64 stream seeded with
    ``seed ^ 0xF1ED``; one draw per non-open qubit in ascending order,
    bit = draw >> 63.
  * 4x4 gate matrices are row-major over the basis |q0 q1>, q0 the high bit.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1

SQRT_X, SQRT_Y, SQRT_W = 0, 1, 2
GATE_NAMES = ("sqrtX", "sqrtY", "sqrtW")


class SplitMix64:
    """splitmix64 (Steele, Lea, Flood 2014; Vigna's public-domain constants)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)


def one_qubit_matrix(kind: int) -> np.ndarray:
    """The three pi/2 rotations about equator axes (paper Sec. 2)."""
    s = 1.0 / math.sqrt(2.0)
    if kind == SQRT_X:
        m = [[1, -1j], [-1j, 1]]
    elif kind == SQRT_Y:
        m = [[1, -1], [1, 1]]
    elif kind == SQRT_W:
        sqrt_i = complex(math.cos(math.pi / 4), math.sin(math.pi / 4))
        sqrt_mi = complex(math.cos(math.pi / 4), -math.sin(math.pi / 4))
        m = [[1, -sqrt_i], [sqrt_mi, 1]]
    else:
        raise ValueError(kind)
    return s * np.array(m, dtype=np.complex128)


def fsim_matrix(theta: float, phi: float) -> np.ndarray:
    """fSim(theta, phi) over |q0 q1> (paper Sec. 2)."""
    c, sn = math.cos(theta), math.sin(theta)
    m = np.zeros((4, 4), dtype=np.complex128)
    m[0, 0] = 1.0
    m[1, 1] = c
    m[1, 2] = -1j * sn
    m[2, 1] = -1j * sn
    m[2, 2] = c
    m[3, 3] = complex(math.cos(phi), -math.sin(phi))
    return m


@dataclass
class Circuit:
    """A gate list.  ``q1[g] < 0`` marks a single-qubit gate whose 2x2 matrix
    sits in ``mats[g, :2, :2]``; otherwise ``mats[g]`` is the 4x4 matrix."""

    n_qubits: int
    q0: np.ndarray          # int32 [n_gates]
    q1: np.ndarray          # int32 [n_gates]
    mats: np.ndarray        # complex128 [n_gates, 4, 4]
    rows: int = 0
    cols: int = 0
    cycles: int = 0
    seed: int = 0
    label: str = ""

    @property
    def n_gates(self) -> int:
        return int(self.q0.shape[0])

    @property
    def n_two_qubit(self) -> int:
        return int((self.q1 >= 0).sum())


@dataclass
class Query:
    """Which amplitudes to compute: every setting of ``open_qubits`` (ascending;
    bit t of the output index is qubit ``open_qubits[t]``) with the other
    qubits pinned to ``fixed_bits[q]``."""

    open_qubits: np.ndarray  # int32 [n_open], ascending
    fixed_bits: np.ndarray   # uint8 [n_qubits]; entries for open qubits are 0

    @property
    def n_open(self) -> int:
        return int(self.open_qubits.shape[0])


@dataclass
class Grid:
    rows: int
    cols: int
    removed: frozenset = field(default_factory=frozenset)

    def qubit_map(self) -> dict:
        qid, k = {}, 0
        for r in range(self.rows):
            for c in range(self.cols):
                if (r, c) in self.removed:
                    continue
                qid[(r, c)] = k
                k += 1
        return qid

    def couplers(self, pattern: int) -> list:
        """Qubit pairs of coupler pattern 0..3 (A, B, C, D)."""
        qid = self.qubit_map()
        pairs = []
        for r in range(self.rows):
            for c in range(self.cols):
                if (r, c) not in qid:
                    continue
                if pattern in (0, 1):
                    if c % 2 == pattern and (r, c + 1) in qid:
                        pairs.append((qid[(r, c)], qid[(r, c + 1)]))
                else:
                    if r % 2 == pattern - 2 and (r + 1, c) in qid:
                        pairs.append((qid[(r, c)], qid[(r + 1, c)]))
        return pairs


def random_circuit(rows: int, cols: int, cycles: int, seed: int,
                   removed=(), theta: float = math.pi / 2,
                   phi: float = math.pi / 6, label: str = "") -> Circuit:
    grid = Grid(rows, cols, frozenset(removed))
    n = len(grid.qubit_map())
    rng = SplitMix64(seed)
    prev = [-1] * n
    q0s, q1s, mats = [], [], []
    fs = fsim_matrix(theta, phi)

    def one_layer():
        for q in range(n):
            u = rng.next() >> 11
            if prev[q] < 0:
                kind = u % 3
            else:
                choices = [g for g in (0, 1, 2) if g != prev[q]]
                kind = choices[u % 2]
            prev[q] = kind
            m = np.zeros((4, 4), dtype=np.complex128)
            m[:2, :2] = one_qubit_matrix(kind)
            q0s.append(q)
            q1s.append(-1)
            mats.append(m)

    for k in range(cycles):
        one_layer()
        for a, b in grid.couplers(k % 4):
            q0s.append(a)
            q1s.append(b)
            mats.append(fs.copy())
    one_layer()
    return Circuit(n, np.array(q0s, dtype=np.int32), np.array(q1s, dtype=np.int32),
                   np.array(mats, dtype=np.complex128), rows, cols, cycles, seed,
                   label or f"{rows}x{cols}-{len(removed)}removed-{cycles}c-s{seed}")


def make_query(n_qubits: int, open_qubits, seed: int) -> Query:
    open_sorted = sorted(int(q) for q in open_qubits)
    if len(set(open_sorted)) != len(open_sorted):
        raise ValueError("open qubits repeat")
    rng = SplitMix64(seed ^ 0xF1ED)
    fixed = np.zeros(n_qubits, dtype=np.uint8)
    oset = set(open_sorted)
    for q in range(n_qubits):
        if q in oset:
            continue
        fixed[q] = rng.next() >> 63
    return Query(np.array(open_sorted, dtype=np.int32), fixed)


# --------------------------------------------------------------------------
# The workloads: small exact case, the 30-qubit sliced case, the 53-qubit
# large-slice case, the batch of uneven circuits and the 40-qubit case.
# --------------------------------------------------------------------------

def grid_12q():
    """3x4 grid, 8 cycles, all 12 qubits open (4096 amplitudes)."""
    c = random_circuit(3, 4, 8, seed=1, label="grid3x4-8c")
    return c, make_query(c.n_qubits, range(12), seed=1)


def grid_30q():
    """5x6 grid, 14 cycles; qubits 20..29 open, 0..19 fixed by seed."""
    c = random_circuit(5, 6, 14, seed=2, label="grid5x6-14c")
    return c, make_query(c.n_qubits, range(20, 30), seed=2)


def grid_53q():
    """6x9 grid minus site (5,8), 12 cycles; the last 12 qubits open."""
    c = random_circuit(6, 9, 12, seed=3, removed=[(5, 8)], label="grid6x9m1-12c")
    return c, make_query(c.n_qubits, range(41, 53), seed=3)


def grid_40q():
    """5x8 grid, 14 cycles; the last 10 qubits open."""
    c = random_circuit(5, 8, 14, seed=5, label="grid5x8-14c")
    return c, make_query(c.n_qubits, range(30, 40), seed=5)


def near_square(n: int):
    r = int(math.isqrt(n))
    cc = -(-n // r)
    removed = []
    extra = r * cc - n
    # remove the last `extra` sites in row-major order
    sites = [(i, j) for i in range(r) for j in range(cc)]
    removed = sites[len(sites) - extra:] if extra else []
    return r, cc, removed


def uneven_batch(count: int = 256, seed: int = 4, n_open: int = 6,
                 n_min: int = 16, n_max: int = 28, c_min: int = 8, c_max: int = 16):
    """``count`` circuits with n ~ U{n_min..n_max} qubits on near-square grids
    and cycles ~ U{c_min..c_max}; the last ``n_open`` qubits open."""
    rng = SplitMix64(seed)
    out = []
    for i in range(count):
        n = n_min + (rng.next() >> 11) % (n_max - n_min + 1)
        cyc = c_min + (rng.next() >> 11) % (c_max - c_min + 1)
        cseed = rng.next()
        r, cc, removed = near_square(n)
        c = random_circuit(r, cc, cyc, seed=cseed, removed=removed,
                           label=f"batch{i}-{n}q-{cyc}c")
        q = make_query(c.n_qubits, range(n - n_open, n), seed=cseed)
        out.append((c, q))
    return out


def small_grid(rows: int, cols: int, cycles: int, seed: int, n_open: int):
    """Any small grid with the last ``n_open`` qubits open (test sizes)."""
    c = random_circuit(rows, cols, cycles, seed=seed)
    n = c.n_qubits
    return c, make_query(n, range(n - n_open, n), seed=seed)
