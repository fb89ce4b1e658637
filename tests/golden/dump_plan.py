"""Record a plan's structure -- its sliced edges and contraction path -- as
data for make_golden.py.  The slice values the oracle computes depend only
on the circuit, the query and the sliced edges (which wires are fixed); the
path only orders the oracle's contraction.  This script runs the library's
host planner (no GPU) with the options the large-slice workload uses.

    python tests/golden/dump_plan.py grid53      # -> grid53_plan.txt

    python tests/golden/dump_plan.py grid30      # -> grid30_plan.txt

Format: "edge q g" lines (slice-id bit j = edge j), "leaf gate qubit" lines
(node i), "step a b" lines (step s makes node n_leaves + s), after a header;
"flops name value" lines carry the planner's flop counts (8 M N K real flops
summed over steps), which the benchmark's oracle arm uses as its unit of work
without loading the library.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import paper_2407_00769_gb300 as tn  # noqa: E402
import rqcgen  # noqa: E402

# the 53-qubit large-slice workload: cap 2^30 elements per slice, one greedy
# trial, 8 slices per pass (the path and edges do not depend on the dtype)
GRID53 = dict(n_slice_edges=-1, max_log2_elems=30, trials=1, slice_batch_log2=3)
# the 30-qubit benchmark workload: 8 sliced edges, 4 greedy restarts, all 256
# slices in one pass (the options bench.py plans it with)
GRID30 = dict(n_slice_edges=8, trials=4, slice_batch_log2=8)


def dump(path, label, plan, opts):
    with open(path, "w") as f:
        f.write(f"# {label}: plan options {opts}\n")
        for q, g in plan.sliced_edges():
            f.write(f"edge {q} {g}\n")
        for g, q in plan.leaf_sources():
            f.write(f"leaf {g} {q}\n")
        for s in plan.steps():
            f.write(f"step {s['a']} {s['b']}\n")
        info = plan.info()
        job = info["flops_per_slice"] * info["n_slices"] + info["flops_invariant"]
        f.write(f"flops per_slice {info['flops_per_slice']!r}\n")
        f.write(f"flops invariant {info['flops_invariant']!r}\n")
        f.write(f"flops job {job!r}\n")


def read(path, with_flops=False):
    edges, leaves, steps, flops = [], [], [], {}
    with open(path) as f:
        for line in f:
            w = line.split()
            if not w or w[0].startswith("#"):
                continue
            if w[0] == "flops":
                flops[w[1]] = float(w[2])
                continue
            v = (int(w[1]), int(w[2]))
            {"edge": edges, "leaf": leaves, "step": steps}[w[0]].append(v)
    return (edges, leaves, steps, flops) if with_flops else (edges, leaves, steps)


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "grid53"
    if what == "grid53":
        c, q = rqcgen.grid_53q()
        p = tn.Plan(c, q, dtype=tn.F16, torch_allocator=False, **GRID53)
        dump(os.path.join(HERE, "grid53_plan.txt"), c.label, p, GRID53)
    elif what == "grid30":
        c, q = rqcgen.grid_30q()
        p = tn.Plan(c, q, dtype=tn.F16, torch_allocator=False, **GRID30)
        dump(os.path.join(HERE, "grid30_plan.txt"), c.label, p, GRID30)
    else:
        raise SystemExit(f"unknown target {what}")
