"""The N > 1 path on CPU: world-size-2 gloo ranks split one plan's slices,
sum their FP64 partials with an all-reduce, and recover the range of a rank
that fails before delivering.  Partials come from the oracle (per-slice
projected state vectors), so no GPU is needed; the host logic is the same
one bench.py uses under torchrun."""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
import rqcgen  # noqa: E402
from paper_2407_00769_gb300 import shard  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case():
    c, q = rqcgen.small_grid(3, 4, 8, seed=12, n_open=5)
    import paper_2407_00769_gb300 as tn
    p = tn.Plan(c, q, dtype=tn.C64, n_slice_edges=3, torch_allocator=False)
    return c, q, p.sliced_edges(), p.info()["n_slices"]


def _worker_allreduce(rank, world, port, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c, q, edges, n = _case()
    b, cnt = shard.slice_range(rank, world, n)
    part = oracle.sliced_amplitudes(c, q, edges, range(b, b + cnt))
    t = torch.from_numpy(part.copy())
    shard.allreduce_amplitudes(t)
    np.save(os.path.join(outdir, f"r{rank}.npy"), t.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_allreduce_equals_full_and_is_rank_ordered(world):
    port = _free_port()
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_worker_allreduce, args=(world, port, d), nprocs=world, join=True)
        c, q, edges, n = _case()
        full = oracle.amplitudes(c, q)
        # the same partials summed in rank order in this process
        parts = []
        for r in range(world):
            b, cnt = shard.slice_range(r, world, n)
            parts.append(oracle.sliced_amplitudes(c, q, edges, range(b, b + cnt)))
        want = shard.ordered_sum(parts)
        for r in range(world):
            got = np.load(os.path.join(d, f"r{r}.npy"))
            assert np.max(np.abs(got - full)) < 1e-13
            # bit-identical on every rank and to the single-process ordered sum
            assert got.tobytes() == want.tobytes()


def _worker_fail(rank, world, port, outdir):
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timeout=__import__("datetime").timedelta(seconds=30))
    c, q, edges, n = _case()
    rng = shard.slice_range(rank, world, n)
    if rank == 1:
        # this rank dies before it delivers anything
        return
    part = oracle.sliced_amplitudes(c, q, edges, range(rng[0], rng[0] + rng[1]))
    shard.publish_partial(store, rank, rng, part)
    got, missing = shard.collect_partials(store, world, 1 << q.n_open, timeout_s=2.0)
    total = shard.recover(n, got, lambda b, k: oracle.sliced_amplitudes(c, q, edges, range(b, b + k)),
                          1 << q.n_open)
    np.save(os.path.join(outdir, "total.npy"), total)
    np.save(os.path.join(outdir, "missing.npy"), np.array(missing))


def test_failed_rank_range_is_recontracted():
    port = _free_port()
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_worker_fail, args=(2, port, d), nprocs=2, join=True)
        c, q, _, _ = _case()
        total = np.load(os.path.join(d, "total.npy"))
        assert np.load(os.path.join(d, "missing.npy")).tolist() == [1]
        assert np.max(np.abs(total - oracle.amplitudes(c, q))) < 1e-13


def test_slice_range_partition_and_uncovered():
    for n in (1, 7, 256):
        for w in (1, 2, 3, 8):
            rs = [shard.slice_range(r, w, n) for r in range(w)]
            assert sum(c for _, c in rs) == n
            assert shard.uncovered(n, rs) == []
            assert all(rs[i][0] + rs[i][1] == rs[i + 1][0] for i in range(w - 1))
    assert shard.uncovered(10, [(0, 3), (5, 2)]) == [(3, 2), (7, 3)]
