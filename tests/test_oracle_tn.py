"""Pins of the FP64 tensor-network oracle (oracle/tn.py) against the
state-vector oracle, which shares none of its arithmetic: the full network
equals the state vector's amplitudes (Sec. 2: both methods compute <x|U|0>),
a slice equals the state vector with the slice's projectors (Sec. 3.1), the
slices of a set of edges sum to the whole, and neither the merge order nor
sub-slicing changes the value."""
import numpy as np
import pytest

import oracle
import rqcgen
from oracle import tn as otn


def _random_order(n_nodes, seed):
    rng = np.random.default_rng(seed)
    live = list(range(n_nodes))
    steps, nxt = [], n_nodes
    while len(live) > 1:
        i, j = rng.choice(len(live), size=2, replace=False)
        a, b = live[i], live[j]
        steps.append((int(a), int(b)))
        live = [x for x in live if x not in (a, b)] + [nxt]
        nxt += 1
    return steps


def _segments_after_two_qubit_gates(c, rng, k):
    segs = []
    for g in range(c.n_gates):
        if c.q1[g] >= 0:
            segs += [(int(c.q0[g]), g), (int(c.q1[g]), g)]
    idx = rng.choice(len(segs), size=k, replace=False)
    return [segs[i] for i in sorted(idx)]


@pytest.mark.parametrize("rows,cols,cycles,n_open,seed", [(2, 3, 5, 6, 1), (3, 3, 6, 4, 2), (3, 4, 6, 5, 3)])
def test_full_network_equals_state_vector(rows, cols, cycles, n_open, seed):
    c, q = rqcgen.small_grid(rows, cols, cycles, seed=seed, n_open=n_open)
    keys = otn.leaf_keys(c)
    want = oracle.amplitudes(c, q)
    for order_seed in range(3):
        got = otn.contract(c, q, keys, _random_order(len(keys), order_seed))
        assert np.max(np.abs(got - want)) <= 1e-13 * max(1.0, np.max(np.abs(want)))


def test_slices_equal_projected_state_vector_and_sum_to_whole():
    c, q = rqcgen.small_grid(3, 3, 6, seed=4, n_open=3)
    keys = otn.leaf_keys(c)
    steps = _random_order(len(keys), 7)
    edges = _segments_after_two_qubit_gates(c, np.random.default_rng(5), 3)
    total = 0
    for s in range(8):
        got = otn.contract(c, q, keys, steps, fixed=otn.slice_fixed(edges, s))
        want = oracle.sliced_amplitudes(c, q, edges, [s])
        assert np.max(np.abs(got - want)) <= 1e-14
        total = total + got
    assert np.max(np.abs(total - oracle.amplitudes(c, q))) <= 1e-13


def test_subslicing_keeps_value_and_bounds_size():
    c, q = rqcgen.small_grid(3, 4, 8, seed=6, n_open=4)
    keys = otn.leaf_keys(c)
    steps = _random_order(len(keys), 3)
    edges = _segments_after_two_qubit_gates(c, np.random.default_rng(2), 2)
    fixed = otn.slice_fixed(edges, 2)
    whole = otn.contract(c, q, keys, steps, fixed=fixed)
    widest = max(len(x) for x in otn._sizes_along(otn._leaf_label_sets(c, q, keys, fixed), steps))
    extra = otn.choose_subslices(c, q, keys, steps, fixed, widest - 2)
    assert 2 <= len(extra) <= 6
    got = otn.contract(c, q, keys, steps, fixed=fixed, max_log2=widest - 2)
    assert np.max(np.abs(got - whole)) <= 1e-14


def test_untouched_qubit_and_all_fixed():
    # qubit 2 has only single-qubit gates: its own group
    m1 = rqcgen.one_qubit_matrix(0)
    f = rqcgen.fsim_matrix(np.pi / 2, np.pi / 6)
    q0 = np.array([0, 2, 0, 1, 2, 1], dtype=np.int32)
    q1 = np.array([-1, -1, 1, -1, -1, 3], dtype=np.int32)
    mats = np.zeros((6, 4, 4), dtype=np.complex128)
    for g in range(6):
        mats[g] = f if q1[g] >= 0 else np.pad(m1, ((0, 2), (0, 2)))
    c = rqcgen.Circuit(n_qubits=4, q0=q0, q1=q1, mats=mats)
    for open_q in ([0, 2], [], [1, 2, 3]):
        fixed_bits = np.zeros(4, dtype=np.uint8)
        fixed_bits[[x for x in range(4) if x not in open_q]] = 1
        fixed_bits[open_q] = 0
        qq = rqcgen.Query(open_qubits=np.array(open_q, dtype=np.int32), fixed_bits=fixed_bits)
        keys = otn.leaf_keys(c)
        assert ("q", 2) in keys
        got = otn.contract(c, qq, keys, _random_order(len(keys), 1))
        want = oracle.amplitudes(c, qq)
        assert np.max(np.abs(got - want)) <= 1e-14
