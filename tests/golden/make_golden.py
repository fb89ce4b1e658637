"""Write oracle-computed expected amplitudes for workloads too large to
recompute inside a test run.  Calls only ``oracle`` (FP64 state vector and
FP64 network contraction) and ``rqcgen`` (inputs); nothing here touches the
GPU library.  The 53-qubit slices read which wires are sliced, and the order
to contract in, from ``grid53_plan.txt`` (data written by dump_plan.py).

    python tests/golden/make_golden.py grid30      # 2^30 state, ~16 GiB RAM
    python tests/golden/make_golden.py grid12      # 3x4 grid, all 4096 amplitudes
    python tests/golden/make_golden.py batch [i0 i1]
    python tests/golden/make_golden.py grid53 [slice ...]   # ~30 min per slice

Output format (text): a header line, then one "index re im" line per
amplitude with 17 significant digits.
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import rqcgen  # noqa: E402


def write(path, label, amps, seconds, method="state-vector"):
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        f.write(f"# {label}: FP64 {method} amplitudes from oracle/ "
                f"({len(amps)} values, {seconds:.0f} s on {oracle.threads()} threads)\n")
        for j, a in enumerate(amps):
            f.write(f"{j} {a.real:.17e} {a.imag:.17e}\n")
    os.replace(tmp, path)


def read(path):
    vals = []
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            _, re, im = line.split()
            vals.append(complex(float(re), float(im)))
    return np.array(vals, dtype=np.complex128)


def grid30():
    c, q = rqcgen.grid_30q()
    t = time.time()
    amps = oracle.amplitudes(c, q)
    write(os.path.join(HERE, "grid5x6_14c_amps.txt"), c.label, amps, time.time() - t)


def grid12():
    c, q = rqcgen.grid_12q()
    t = time.time()
    amps = oracle.amplitudes(c, q)
    write(os.path.join(HERE, "grid3x4_8c_amps.txt"), c.label, amps, time.time() - t)


def batch(i0=0, i1=256):
    items = rqcgen.uneven_batch()
    for i in range(i0, i1):
        c, q = items[i]
        path = os.path.join(HERE, "batch", f"circuit{i:03d}.txt")
        if os.path.exists(path):
            continue
        os.makedirs(os.path.dirname(path), exist_ok=True)
        t = time.time()
        amps = oracle.amplitudes(c, q)
        write(path, c.label, amps, time.time() - t)


def grid53(slices=(0,)):
    import dump_plan
    from oracle import tn as otn
    c, q = rqcgen.grid_53q()
    edges, leaves, steps = dump_plan.read(os.path.join(HERE, "grid53_plan.txt"))
    keys = [("g", g) if g >= 0 else ("q", qq) for g, qq in leaves]
    for sid in slices:
        path = os.path.join(HERE, f"grid53_slice{sid}.txt")
        t = time.time()
        # sub-sliced to 2^29 entries per intermediate (8 GiB in FP64)
        amps = otn.contract(c, q, keys, steps, fixed=otn.slice_fixed(edges, sid), max_log2=29)
        write(path, f"{c.label} slice {sid} of the sliced edges in grid53_plan.txt", amps,
              time.time() - t, method="tensor-network")


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "grid30"
    if what == "grid30":
        grid30()
    elif what == "grid12":
        grid12()
    elif what == "batch":
        a = [int(x) for x in sys.argv[2:4]] or [0, 256]
        batch(*a)
    elif what == "grid53":
        sys.path.insert(0, HERE)
        grid53([int(x) for x in sys.argv[2:]] or [0])
    else:
        raise SystemExit(f"unknown target {what}")
