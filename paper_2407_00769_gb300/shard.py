"""Splitting the slices of one plan across ranks (one process per GPU).

Slices are independent sub-networks (paper Sec. 3.1, global level), so rank r
of N contracts the contiguous range ``slice_range(r, N, S)`` with no data
exchange, and the FP64 partial amplitude vectors are summed once at the end
(``allreduce_amplitudes``: every rank gathers all partials, at most 2^12
complex128 each, and adds them in rank order, so every rank holds the same
bits, equal to the single-process sum of the same partials in the same
order).  Because a slice range is idempotent, a range that a failed rank
never delivered can simply be contracted again by a surviving rank: ``collect_partials`` publishes each
rank's partial sum through a torch.distributed store, rank 0 waits for them
with a deadline and reports the ranges that never arrived.
"""
from __future__ import annotations

import time
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np


def slice_range(rank: int, world: int, n_slices: int) -> Tuple[int, int]:
    """(begin, count) of rank's share: contiguous, sizes differing by <= 1."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    b = rank * n_slices // world
    e = (rank + 1) * n_slices // world
    return b, e - b


def uncovered(n_slices: int, done: Sequence[Tuple[int, int]]) -> List[Tuple[int, int]]:
    """Ranges of [0, n_slices) not covered by the (begin, count) list."""
    marks = np.zeros(n_slices + 1, dtype=np.int64)
    for b, c in done:
        if c <= 0:
            continue
        marks[b] += 1
        marks[b + c] -= 1
    cov = np.cumsum(marks[:-1]) > 0
    out, i = [], 0
    while i < n_slices:
        if not cov[i]:
            j = i
            while j < n_slices and not cov[j]:
                j += 1
            out.append((i, j - i))
            i = j
        else:
            i += 1
    return out


def allreduce_amplitudes(amps, group=None):
    """Sum complex128 amplitude tensors over all ranks, in place, in fixed
    rank order: the partials are all-gathered (one collective) and every rank
    adds them as ((p_0 + p_1) + p_2) + ...  An all-reduce would leave the
    order of the additions to the collective's algorithm; this order makes
    the result bit-identical on every rank, from run to run and to the
    ordered sum ``ordered_sum`` of the same partials in one process."""
    import torch
    import torch.distributed as dist
    if amps.dtype != torch.complex128:
        raise ValueError("amplitudes must be complex128")
    if not amps.is_contiguous():
        raise ValueError("amplitudes must be contiguous")
    world = dist.get_world_size(group)
    flat = torch.view_as_real(amps).reshape(-1)
    parts = [torch.empty_like(flat) for _ in range(world)]
    dist.all_gather(parts, flat, group=group)
    flat.copy_(parts[0])
    for p in parts[1:]:
        flat.add_(p)
    return amps


def ordered_sum(partials):
    """The rank-ordered sum that ``allreduce_amplitudes`` computes, for
    partials held in one process (a list of complex128 arrays)."""
    total = np.array(partials[0], dtype=np.complex128, copy=True)
    for p in partials[1:]:
        total += np.asarray(p, dtype=np.complex128)
    return total


def publish_partial(store, rank: int, rng: Tuple[int, int], partial: np.ndarray) -> None:
    """Make rank's partial amplitude sum over ``rng`` visible to rank 0."""
    arr = np.ascontiguousarray(partial, dtype=np.complex128)
    store.set(f"tn/partial/{rank}", arr.tobytes())
    store.set(f"tn/range/{rank}", f"{rng[0]},{rng[1]}")


def collect_partials(store, world: int, n_amps: int, timeout_s: float,
                     poll_s: float = 0.05) -> Tuple[Dict[int, Tuple[Tuple[int, int], np.ndarray]], List[int]]:
    """Rank 0: gather every published partial until ``timeout_s``; return
    {rank: (range, partial)} and the ranks that never delivered."""
    got: Dict[int, Tuple[Tuple[int, int], np.ndarray]] = {}
    deadline = time.monotonic() + timeout_s
    pending = set(range(world))
    while pending and time.monotonic() < deadline:
        for r in sorted(pending):
            key = f"tn/range/{r}"
            if store.check([key]):
                b, c = (int(x) for x in store.get(key).decode().split(","))
                buf = store.get(f"tn/partial/{r}")
                got[r] = ((b, c), np.frombuffer(buf, dtype=np.complex128, count=n_amps).copy())
                pending.discard(r)
        if pending:
            time.sleep(poll_s)
    return got, sorted(pending)


def recover(n_slices: int, got: Dict[int, Tuple[Tuple[int, int], np.ndarray]], contract_range,
            n_amps: int) -> np.ndarray:
    """Sum the delivered partials and contract every missing range again with
    ``contract_range(begin, count) -> partial``.  Ranges are summed in
    ascending order of their first slice."""
    parts = [(rng, p) for rng, p in got.values()]
    for rng in uncovered(n_slices, [rng for rng, _ in parts]):
        parts.append((rng, np.asarray(contract_range(*rng), dtype=np.complex128)))
    total = np.zeros(n_amps, dtype=np.complex128)
    for _, p in sorted(parts, key=lambda x: x[0][0]):
        total += p
    return total
