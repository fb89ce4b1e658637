"""FP64 tensor-network contraction of slices -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` and the scripts under ``tests/golden/`` use this module; it
never imports the GPU library.  It is the network method of Sec. 2 (the
circuit read as a tensor network whose full contraction gives the queried
amplitudes) with the slicing of Sec. 3.1 (fixing the value of chosen edges
splits the network into independent sub-networks whose sum is the whole),
written plainly in numpy, FP64:

* one tensor per circuit element: |0> at the start of every wire, every gate
  (2x2 as [out, in], 4x4 as [out0, out1, in0, in1] with basis |q0 q1>, q0 the
  high bit), <x_q| at the end of every fixed wire; an open qubit's last wire
  segment stays an open index.  Wire segment (q, g) is the wire of qubit q
  right after gate g; (q, -1) starts at |0>.
* a slice fixes segments: segment (q, g) at value b keeps index b on both
  tensors that carry it, i.e. the projector |b><b| on that wire right after
  gate g.  Slice id bit j (LSB first) is the value of sliced segment j.
* tensors are grouped, one group per two-qubit gate (with the single-qubit
  gates before it on its wires, and the start vectors or output vectors of
  wires it opens or closes), one group per qubit that no two-qubit gate
  touches; the groups are then merged pairwise in a given order, each merge
  one ``np.tensordot`` over the labels the two share.
* ``max_log2``: further segments are fixed ("sub-slicing") until every
  intermediate holds at most 2^max_log2 entries, and the sub-slices summed.

The merge order is data: every order gives the same value up to rounding and
only sets the cost, which the tests check by contracting the same network in
random orders and against the state vector.
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np


def _elements(circuit, query):
    """[(labels, array)] and the open labels in output-bit order."""
    n = int(circuit.n_qubits)
    cur = [(q, -1) for q in range(n)]                  # current segment per wire
    els = []
    for q in range(n):
        els.append(([(q, -1)], np.array([1.0, 0.0], dtype=np.complex128)))
    for g in range(circuit.n_gates):
        a, b = int(circuit.q0[g]), int(circuit.q1[g])
        m = np.asarray(circuit.mats[g], dtype=np.complex128)
        if b < 0:
            els.append(([(a, g), cur[a]], m[:2, :2].copy()))
            cur[a] = (a, g)
        else:
            els.append(([(a, g), (b, g), cur[a], cur[b]], m.reshape(2, 2, 2, 2).copy()))
            cur[a], cur[b] = (a, g), (b, g)
    open_set = set(int(x) for x in query.open_qubits)
    for q in range(n):
        if q not in open_set:
            v = np.zeros(2, dtype=np.complex128)
            v[int(query.fixed_bits[q])] = 1.0
            els.append(([cur[q]], v))
    open_labels = [cur[int(q)] for q in query.open_qubits]
    return els, open_labels


def leaf_keys(circuit) -> List[Tuple[str, int]]:
    """The groups in a canonical order: two-qubit gates in circuit order, then
    untouched qubits ascending."""
    keys = [("g", g) for g in range(circuit.n_gates) if int(circuit.q1[g]) >= 0]
    touched = set()
    for g in range(circuit.n_gates):
        if int(circuit.q1[g]) >= 0:
            touched.add(int(circuit.q0[g]))
            touched.add(int(circuit.q1[g]))
    keys += [("q", q) for q in range(int(circuit.n_qubits)) if q not in touched]
    return keys


def _group_of_elements(circuit, query):
    """Group key of every element of ``_elements`` (same order)."""
    n = int(circuit.n_qubits)
    two = [[] for _ in range(n)]              # two-qubit gate indices per wire
    for g in range(circuit.n_gates):
        if int(circuit.q1[g]) >= 0:
            two[int(circuit.q0[g])].append(g)
            two[int(circuit.q1[g])].append(g)

    def nxt(q, g):                            # first two-qubit gate on q after g
        for t in two[q]:
            if t > g:
                return ("g", t)
        return ("g", two[q][-1]) if two[q] else ("q", q)

    keys = [nxt(q, -1) for q in range(n)]     # start vectors
    for g in range(circuit.n_gates):
        if int(circuit.q1[g]) >= 0:
            keys.append(("g", g))
        else:
            keys.append(nxt(int(circuit.q0[g]), g))
    open_set = set(int(x) for x in query.open_qubits)
    for q in range(n):
        if q not in open_set:
            keys.append(("g", two[q][-1]) if two[q] else ("q", q))
    return keys


def _fix(labels, arr, fixed: Dict):
    """Take index fixed[l] on every axis whose label is fixed."""
    keep = []
    for l in labels:
        if l in fixed:
            arr = np.take(arr, fixed[l], axis=len(keep))
        else:
            keep.append(l)
    return keep, arr


def _merge(la, a, lb, b):
    """Contract two tensors over their shared labels (np.tensordot)."""
    shared = [l for l in la if l in lb]
    ia = [la.index(l) for l in shared]
    ib = [lb.index(l) for l in shared]
    out = np.tensordot(a, b, axes=(ia, ib))
    return [l for l in la if l not in shared] + [l for l in lb if l not in shared], out


def _leaf_label_sets(circuit, query, keys, fixed):
    els, _ = _elements(circuit, query)
    gk = _group_of_elements(circuit, query)
    sets = {k: [] for k in keys}
    for (labels, _), k in zip(els, gk):
        for l in labels:
            if l in fixed:
                continue
            if l in sets[k]:
                sets[k].remove(l)             # internal to the group
            else:
                sets[k].append(l)
    return [sets[k] for k in keys]


def _sizes_along(leaf_sets, steps):
    """Label sets of every intermediate along the merge order."""
    nodes = [list(s) for s in leaf_sets]
    out = []
    for a, b in steps:
        la, lb = nodes[a], nodes[b]
        res = [l for l in la if l not in lb] + [l for l in lb if l not in la]
        nodes.append(res)
        out.append(res)
    return out


def choose_subslices(circuit, query, keys, steps, fixed, max_log2: int):
    """Segments to fix in addition to ``fixed`` so that every intermediate
    has at most max_log2 labels: repeatedly the summed-over segment carried by
    the most oversized intermediates (ties: smallest segment)."""
    extra = []
    fx = dict(fixed)
    _, open_labels = _elements(circuit, query)
    never = set(open_labels)                  # output indices are not summed over
    while True:
        leaf_sets = _leaf_label_sets(circuit, query, keys, fx)
        inter = _sizes_along(leaf_sets, steps) + leaf_sets
        big = [s for s in inter if len(s) > max_log2]
        if not big:
            return extra
        count = {}
        for s in big:
            for l in s:
                if l not in never:
                    count[l] = count.get(l, 0) + 1
        if not count:
            raise ValueError("max_log2 is below the number of open indices")
        best = min(count, key=lambda l: (-count[l], l))
        extra.append(best)
        fx[best] = 0


def contract(circuit, query, keys: Sequence[Tuple[str, int]], steps: Sequence[Tuple[int, int]],
             fixed: Optional[Dict] = None, max_log2: Optional[int] = None) -> np.ndarray:
    """Amplitudes (2^n_open complex128, bit t of the index = open qubit t) of
    the network with the segments in ``fixed`` ({(q, g): bit}) fixed.

    ``keys[i]`` is the group of node i (("g", gate) or ("q", qubit));
    ``steps[s] = (a, b)`` merges nodes a and b into node len(keys) + s."""
    fixed = dict(fixed or {})
    extra = choose_subslices(circuit, query, keys, steps, fixed, max_log2) if max_log2 else []
    els, open_labels = _elements(circuit, query)
    gk = _group_of_elements(circuit, query)
    pos = {k: i for i, k in enumerate(keys)}
    if len(pos) != len(keys) or any(k not in pos for k in gk):
        raise ValueError("group keys do not cover the circuit")
    total = None
    for bits in itertools.product((0, 1), repeat=len(extra)):
        fx = dict(fixed)
        fx.update({l: b for l, b in zip(extra, bits)})
        nodes: List = [None] * len(keys)
        for (labels, arr), k in zip(els, gk):
            la, a = _fix(labels, arr, fx)
            i = pos[k]
            nodes[i] = (la, a) if nodes[i] is None else _merge(nodes[i][0], nodes[i][1], la, a)
        for a, b in steps:
            (la, ta), (lb, tb) = nodes[a], nodes[b]
            nodes.append(_merge(la, ta, lb, tb))
            nodes[a] = nodes[b] = None
        rest = [x for x in nodes if x is not None]
        labels, arr = rest[0]
        for lb, tb in rest[1:]:                  # disconnected parts: outer product
            labels, arr = _merge(labels, arr, lb, tb)
        # axis order: open qubit t at bit t, i.e. the last open qubit outermost
        order = [labels.index(l) for l in reversed(open_labels)]
        amp = np.transpose(arr, order).reshape(-1) if order else arr.reshape(1)
        total = amp.copy() if total is None else total + amp
    return total


def slice_fixed(sliced_edges: Sequence[Tuple[int, int]], slice_id: int) -> Dict:
    """{(qubit, after_gate): bit} of one slice; bit j of slice_id fixes edge j."""
    return {(int(q), int(g)): (int(slice_id) >> j) & 1 for j, (q, g) in enumerate(sliced_edges)}
