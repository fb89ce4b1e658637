"""Collect autotuner timings for the learned cost model's training set.

Exhaustively tunes plans of the 12-qubit, 30-qubit and 53-qubit workloads
(several slice batchings, complex-half dtypes, greedy and annealed paths)
on the current GPU and writes every timing the tuner takes -- GEMM steps
with each legal (kernel, tile) and permutations -- to an .npz file:

    python -m paper_2407_00769_gb300.data.collect_timings [out.npz] [minutes]

Fields: kind, lm, ln, lk, lb, dtype, kernel, tile, ms (one entry per
timing) and label (the plan each came from).
"""
import itertools
import os
import sys
import time

import numpy as np

FIELDS = ("kind", "lm", "ln", "lk", "lb", "dtype", "kernel", "tile")


def plan_configs():
    import rqcgen
    import paper_2407_00769_gb300 as tn
    dts = (tn.F16, tn.BF16)
    c12, q12 = rqcgen.grid_12q()
    c30, q30 = rqcgen.grid_30q()
    c53, q53 = rqcgen.grid_53q()
    for dt, b in itertools.product(dts, (0,)):
        yield f"grid12 dt{dt}", c12, q12, dict(dtype=dt, n_slice_edges=2, slice_batch_log2=b)
    for ann, dt, b in itertools.product((0, 200000), dts, (8, 6, 4, 2, 0)):
        yield (f"grid30 anneal{ann} dt{dt} b{b}", c30, q30,
               dict(dtype=dt, n_slice_edges=8, trials=4, slice_batch_log2=b, anneal_iters=ann))
    for ann, cap, b in itertools.product((200000, 0), (28, 30), (3, 1)):
        yield (f"grid53 anneal{ann} cap{cap} b{b}", c53, q53,
               dict(dtype=tn.F16, n_slice_edges=-1, max_log2_elems=cap, trials=1, slice_batch_log2=b,
                    anneal_iters=ann))
    for cap, ann, b in itertools.product((20, 22, 24, 26), (0, 200000), (4, 0)):
        yield (f"grid30 cap{cap} anneal{ann} b{b}", c30, q30,
               dict(dtype=tn.F16, n_slice_edges=-1, max_log2_elems=cap, trials=4, slice_batch_log2=b,
                    anneal_iters=ann))
    for cap, ann, b in itertools.product((24, 26), (200000, 0), (3, 0)):
        yield (f"grid53 cap{cap} anneal{ann} b{b}", c53, q53,
               dict(dtype=tn.F16, n_slice_edges=-1, max_log2_elems=cap, trials=1, slice_batch_log2=b,
                    anneal_iters=ann))
    for seed, b in itertools.product(range(1, 17), (3, 0)):
        c, q = rqcgen.small_grid(4 + seed % 2, 5, 10 + seed % 8, seed=100 + seed, n_open=6)
        yield f"small seed{seed} b{b}", c, q, dict(dtype=tn.F16, n_slice_edges=4, slice_batch_log2=b)


def main():
    import torch
    import paper_2407_00769_gb300 as tn
    out = sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(__file__), "timings_gb300.npz")
    budget = float(sys.argv[2]) * 60 if len(sys.argv) > 2 else 12 * 60
    cols = {f: [] for f in FIELDS + ("ms", "label")}
    labels = []
    t0 = time.time()
    for label, c, q, kw in plan_configs():
        if time.time() - t0 > budget:
            break
        try:
            p = tn.Plan(c, q, **kw)
            p.tune()
            recs = p.tune_records()
        except tn.TnError as e:
            print(f"{label}: skipped ({e})", flush=True)
            continue
        finally:
            p = None
            torch.cuda.empty_cache()
        li = len(labels)
        labels.append(label)
        for r in recs:
            for f in FIELDS:
                cols[f].append(r[f])
            cols["ms"].append(r["ms"])
            cols["label"].append(li)
        print(f"{label}: {len(recs)} timings, total {len(cols['ms'])}, {time.time() - t0:.0f} s", flush=True)
    arrays = {f: np.array(cols[f], dtype=np.int32) for f in FIELDS + ("label",)}
    arrays["ms"] = np.array(cols["ms"], dtype=np.float64)
    arrays["labels"] = np.array(labels)
    arrays["gpu"] = np.array(torch.cuda.get_device_name(0))
    np.savez_compressed(out, **arrays)
    print(f"wrote {out}: {len(cols['ms'])} timings from {len(labels)} plans", flush=True)


if __name__ == "__main__":
    main()
