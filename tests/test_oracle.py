"""Pins of the FP64 oracle against facts that do not come from the oracle:
closed forms, unitarity, brute force, the paper's worked example, and
invariants (norm, slice sum = whole)."""
import math
import os

import numpy as np
import pytest

import oracle
import rqcgen

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            vals[k.strip()] = v.split()
    return vals


def _layer_circuit(n, kind):
    m = np.zeros((n, 4, 4), dtype=np.complex128)
    for q in range(n):
        m[q, :2, :2] = rqcgen.one_qubit_matrix(kind)
    return rqcgen.Circuit(n, np.arange(n, dtype=np.int32), -np.ones(n, dtype=np.int32), m)


def _custom(n, gates):
    q0 = np.array([g[0] for g in gates], dtype=np.int32)
    q1 = np.array([g[1] for g in gates], dtype=np.int32)
    mats = np.zeros((len(gates), 4, 4), dtype=np.complex128)
    for i, g in enumerate(gates):
        mat = np.asarray(g[2], dtype=np.complex128)
        mats[i, :mat.shape[0], :mat.shape[1]] = mat
    return rqcgen.Circuit(n, q0, q1, mats)


def test_splitmix64_published_vector():
    want = [int(x, 16) for x in _read_golden("splitmix64.txt")["seed0"]]
    r = rqcgen.SplitMix64(0)
    assert [r.next() for _ in want] == want


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_one_qubit_gates_unitary(kind):
    m = rqcgen.one_qubit_matrix(kind)
    assert np.allclose(m.conj().T @ m, np.eye(2), atol=1e-15)


def test_fsim_unitary_and_symmetric():
    f = rqcgen.fsim_matrix(math.pi / 2, math.pi / 6)
    assert np.allclose(f.conj().T @ f, np.eye(4), atol=1e-15)
    swap = np.eye(4)[[0, 2, 1, 3]]
    assert np.allclose(swap @ f @ swap, f)  # symmetric under qubit exchange


@pytest.mark.parametrize("n", [3, 7, 12])
def test_sqrt_y_layer_uniform(n):
    # sqrt(Y)|0> = (|0> + |1>)/sqrt2: every amplitude is 2^{-n/2}
    psi = oracle.state_vector(_layer_circuit(n, rqcgen.SQRT_Y))
    assert np.allclose(psi, 2.0 ** (-n / 2), atol=1e-14)


@pytest.mark.parametrize("n", [4, 9])
def test_sqrt_x_and_sqrt_w_layer_closed_form(n):
    idx = np.arange(1 << n)
    pop = np.array([bin(i).count("1") for i in idx])
    psi = oracle.state_vector(_layer_circuit(n, rqcgen.SQRT_X))
    assert np.allclose(psi, (-1j) ** pop * 2.0 ** (-n / 2), atol=1e-14)
    psi = oracle.state_vector(_layer_circuit(n, rqcgen.SQRT_W))
    assert np.allclose(psi, np.exp(-1j * math.pi / 4 * pop) * 2.0 ** (-n / 2), atol=1e-14)


def test_hadamard_layer_uniform():
    h = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    n = 10
    psi = oracle.state_vector(_custom(n, [(q, -1, h) for q in range(n)]))
    assert np.allclose(psi, 2.0 ** (-n / 2), atol=1e-14)


def test_fsim_on_basis_states_closed_form():
    # X on chosen qubits prepares a basis state; fSim(pi/2, phi) maps
    # |01> -> -i|10>, |10> -> -i|01>, |11> -> e^{-i phi}|11>, |00> -> |00>.
    n, phi = 8, math.pi / 6
    x = np.array([[0, 1], [1, 0]])
    bits = [1, 0, 0, 1, 1, 1, 0, 0]
    pairs = [(0, 1), (2, 3), (4, 5), (6, 7)]
    gates = [(q, -1, x) for q in range(n) if bits[q]]
    gates += [(a, b, rqcgen.fsim_matrix(math.pi / 2, phi)) for a, b in pairs]
    psi = oracle.state_vector(_custom(n, gates))
    out, phase = list(bits), 1.0 + 0j
    for a, b in pairs:
        if bits[a] != bits[b]:
            out[a], out[b] = bits[b], bits[a]
            phase *= -1j
        elif bits[a] == 1:
            phase *= np.exp(-1j * phi)
    k = sum(v << q for q, v in enumerate(out))
    want = np.zeros(1 << n, dtype=np.complex128)
    want[k] = phase
    assert np.allclose(psi, want, atol=1e-15)


def test_two_qubit_basis_order_q0_high():
    # CNOT with control on the high bit of |q0 q1>: control q0, target q1.
    cnot = np.eye(4)[[0, 1, 3, 2]]
    x = np.array([[0, 1], [1, 0]])
    n = 5
    psi = oracle.state_vector(_custom(n, [(3, -1, x), (3, 1, cnot)]))
    k = (1 << 3) | (1 << 1)
    assert abs(psi[k] - 1) < 1e-15 and np.count_nonzero(np.abs(psi) > 1e-15) == 1
    psi = oracle.state_vector(_custom(n, [(3, -1, x), (1, 3, cnot)]))  # control 1 is |0>
    assert abs(psi[1 << 3] - 1) < 1e-15


@pytest.mark.parametrize("rows,cols,cycles", [(2, 3, 6), (2, 4, 8), (1, 5, 5)])
def test_state_vector_equals_bruteforce(rows, cols, cycles):
    c = rqcgen.random_circuit(rows, cols, cycles, seed=11 + rows * cols)
    a = oracle.state_vector(c)
    b = oracle.bruteforce_state(c)
    assert np.max(np.abs(a - b)) < 1e-13


@pytest.mark.parametrize("rows,cols,cycles,seed", [(3, 4, 8, 1), (4, 5, 10, 9)])
def test_norm_is_one(rows, cols, cycles, seed):
    c = rqcgen.random_circuit(rows, cols, cycles, seed=seed)
    psi = oracle.state_vector(c)
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-12


def test_projectors_sum_to_identity():
    # sum over all slices of the wire-projected evolutions = the full result,
    # and each single slice is a strict part of it
    c, q = rqcgen.small_grid(3, 3, 6, seed=5, n_open=4)
    two_q = np.nonzero(c.q1 >= 0)[0]
    edges = [(int(c.q0[two_q[3]]), int(two_q[3])), (int(c.q1[two_q[7]]), int(two_q[7])),
             (int(c.q0[two_q[12]]), int(two_q[12]))]
    full = oracle.amplitudes(c, q)
    total = oracle.sliced_amplitudes(c, q, edges, range(1 << len(edges)))
    assert np.max(np.abs(total - full)) < 1e-14
    one = oracle.amplitudes(c, q, oracle.slice_projectors(edges, 5))
    assert oracle.rel_l2(one, full) > 0.05


def test_gather_bit_order():
    c, q = rqcgen.small_grid(2, 3, 4, seed=3, n_open=3)
    psi = oracle.state_vector(c)
    amps = oracle.gather(c, q, psi)
    for j in range(8):
        x = sum(int(q.fixed_bits[k]) << k for k in range(c.n_qubits) if k not in q.open_qubits)
        for t, oq in enumerate(q.open_qubits):
            x |= ((j >> t) & 1) << int(oq)
        assert amps[j] == psi[x]


def test_complex_half_einsum_worked_example():
    g = _read_golden("complex_half_example.txt")
    a = np.array([float(v) for v in g["A_complex"]]).reshape(2, 2)  # modes a1, a2(re/im)
    b = np.array([float(v) for v in g["B_complex"]])
    bc = np.array([b[0] + 1j * b[1]])                               # mode b1 (dim 1)
    bp = oracle.pad_b(bc)                                           # modes c0, b1, a2
    assert np.array_equal(bp.reshape(2, 2), np.array([float(v) for v in g["B_padded"]]).reshape(2, 2))
    c = oracle.complex_as_real_einsum("a,b->ab", a, bc)             # modes a1, b1, c0
    want = np.array([float(v) for v in g["C_complex"]]).reshape(2, 1, 2)
    assert np.array_equal(c, want)


def test_complex_half_einsum_matches_complex_einsum():
    rng = np.random.default_rng(7)
    a = rng.normal(size=(4, 2, 8)) + 1j * rng.normal(size=(4, 2, 8))
    b = rng.normal(size=(8, 2, 3)) + 1j * rng.normal(size=(8, 2, 3))
    a_real = np.stack([a.real, a.imag], axis=-1)
    c = oracle.complex_as_real_einsum("mjk,kjn->mn", a_real, b)
    want = np.einsum("mjk,kjn->mn", a, b)
    assert np.allclose(c[..., 0] + 1j * c[..., 1], want, atol=1e-12)


def test_metrics():
    rng = np.random.default_rng(3)
    b = rng.normal(size=64) + 1j * rng.normal(size=64)
    assert oracle.rel_l2(b, b) == 0.0
    assert abs(oracle.fidelity(b, (0.3 - 2j) * b) - 1.0) < 1e-12
    o = np.zeros(64, complex); o[0] = 1
    e = np.zeros(64, complex); e[1] = 1j
    assert oracle.fidelity(o, e) == 0.0
    assert abs(oracle.fidelity(o + e, o) - 0.5) < 1e-15
    # uniform distribution has XEB 0; a delta on the support of size 1 has 2^n - 1
    assert abs(oracle.linear_xeb(np.full(8, 1 / 16), 4)) < 1e-15
    idx, p = oracle.topk(np.array([1, 2, -2, 0.5, 2j]), 3)
    assert list(idx) == [1, 2, 4] and np.allclose(p, 4)


def test_porter_thomas_sanity():
    # deep random circuit: 2^n |amp|^2 over a 2^10 subspace ~ Exp(1)
    c, q = rqcgen.small_grid(4, 5, 14, seed=21, n_open=10)
    amps = oracle.amplitudes(c, q)
    x = (1 << c.n_qubits) * np.abs(amps) ** 2
    assert 0.8 < x.mean() < 1.2 and 0.6 < x.var() < 1.6


def test_projector_acts_right_after_its_gate():
    # gate 0 prepares 0.6|0> + 0.8|1>, gate 1 is X.  Fixing the wire to 1
    # after gate 0 leaves 0.8|1> -> X -> 0.8|0>; after gate 1 it leaves 0.6|1>;
    # before gate 0 (wire still |0>) it leaves nothing.
    prep = np.array([[0.6, -0.8], [0.8, 0.6]])
    x = np.array([[0, 1], [1, 0]])
    c = _custom(2, [(0, -1, prep), (0, -1, x)])
    assert np.allclose(oracle.state_vector(c, [(0, 0, 1)]), [0.8, 0, 0, 0], atol=1e-15)
    assert np.allclose(oracle.state_vector(c, [(0, 1, 1)]), [0, 0.6, 0, 0], atol=1e-15)
    assert np.allclose(oracle.state_vector(c, [(0, -1, 1)]), [0, 0, 0, 0], atol=1e-15)


def test_slice_bits_lsb_first():
    assert oracle.slice_projectors([(0, 5), (1, 6), (4, 9)], 6) == [(0, 5, 0), (1, 6, 1), (4, 9, 1)]


def test_stored_grid12_amplitudes_are_the_oracles():
    # the stored 12-qubit amplitudes (read by the benchmark's latency leg)
    # are the oracle's, and form a whole normalised state
    rows = [l.split() for l in open(os.path.join(GOLD, "grid3x4_8c_amps.txt")) if not l.startswith("#")]
    stored = np.array([complex(float(r[1]), float(r[2])) for r in rows])
    c, q = rqcgen.grid_12q()
    assert np.allclose(stored, oracle.amplitudes(c, q), rtol=0, atol=1e-15)
    assert abs(np.vdot(stored, stored).real - 1.0) < 1e-12


def test_oracle_and_product_share_no_code():
    # the oracle is the independent check of the CUDA path: neither side may
    # import, include or link the other (the seeded input generators in
    # rqcgen serve both and hold none of the method's arithmetic)
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_2407_00769_gb300")
    orc = os.path.join(root, "oracle")

    def sources(top, exts):
        for d, dirs, files in os.walk(top):
            dirs[:] = [x for x in dirs if x not in ("_build", "__pycache__")]
            for f in files:
                if f.endswith(exts):
                    yield os.path.join(d, f)

    imports_oracle = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b)|#include\s+[\"<][^\">]*oracle", re.M)
    for path in sources(pkg, (".py", ".cu", ".cuh", ".cpp", ".h")):
        assert not imports_oracle.search(open(path).read()), path
    imports_pkg = re.compile(r"^\s*(import\s+paper_2407_00769_gb300|from\s+paper_2407_00769_gb300\b)"
                             r"|#include\s+[\"<][^\">]*(tn\.h|csrc)", re.M)
    for path in sources(orc, (".py", ".c", ".h")):
        assert not imports_pkg.search(open(path).read()), path
    src = open(os.path.join(root, "rqcgen", "__init__.py")).read()
    assert not re.search(r"^\s*(import|from)\s+(oracle|paper_2407_00769_gb300)\b", src, re.M)
