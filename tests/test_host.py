"""Host-side checks of the library that need no GPU: it loads, exports every
symbol include/tn.h declares, and its planner obeys the paper's GEMM
condition (Sec. 3.3: reduced modes = shared modes, stated after Eq. 3; result modes, Eq. 4) and the slicing/memory invariants."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import rqcgen
import paper_2407_00769_gb300 as tn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "tn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tn_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = tn.lib()
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(L, s), s
    assert set(syms) == set(tn.EXPORTED)


def test_strerror_codes():
    L = tn.lib()
    assert L.tn_strerror(0) == b"ok"
    assert L.tn_strerror(4) == b"device wait timed out"


def _plan(circuit, query, **kw):
    kw.setdefault("torch_allocator", False)
    return tn.Plan(circuit, query, **kw)


@pytest.mark.parametrize("dtype", [tn.C64, tn.F16])
@pytest.mark.parametrize("slices,batch", [(0, 0), (3, 0), (3, 2)])
def test_plan_steps_are_pure_gemms(dtype, slices, batch):
    # Eq. 3-4: every step's result has exactly the modes of A and B minus the
    # reduced ones; the sizes each tensor is produced with and consumed with
    # must agree, and the last tensor holds the open modes (+ batch modes).
    c, q = rqcgen.small_grid(4, 4, 10, seed=3, n_open=5)
    p = _plan(c, q, dtype=dtype, n_slice_edges=slices, slice_batch_log2=batch)
    info = p.info()
    steps = p.steps()
    assert info["n_steps"] == info["n_leaves"] - 1 == len(steps)
    size = {}
    for s in steps:
        la = s["log2_batch"] + s["log2_m"] + s["log2_k"]
        lb = s["log2_batch"] + s["log2_k"] + s["log2_n"]
        for t, l in ((s["a"], la), (s["b"], lb)):
            if t in size:
                assert size[t] == l
        size[s["c"]] = s["log2_batch"] + s["log2_m"] + s["log2_n"]
        assert size[s["c"]] <= info["max_log2_elems"] + batch
        # A is the larger operand
        assert la >= lb
    assert size[steps[-1]["c"]] == info["n_open"] + batch


def test_slicing_hits_count_and_reduces_width():
    c, q = rqcgen.small_grid(4, 5, 12, seed=4, n_open=6)
    w0 = _plan(c, q, n_slice_edges=0).info()["max_log2_elems"]
    for s in (1, 3, 5):
        i = _plan(c, q, n_slice_edges=s).info()
        assert i["n_slice_edges"] == s and i["n_slices"] == 1 << s
        assert i["max_log2_elems"] <= w0


def test_cap_mode_reaches_cap():
    c, q = rqcgen.small_grid(4, 5, 12, seed=4, n_open=6)
    w0 = _plan(c, q, n_slice_edges=0).info()["max_log2_elems"]
    cap = w0 - 3
    i = _plan(c, q, n_slice_edges=-1, max_log2_elems=cap).info()
    assert i["max_log2_elems"] <= cap and i["n_slice_edges"] >= 1


def test_sliced_edges_are_two_qubit_wires():
    c, q = rqcgen.small_grid(4, 4, 10, seed=3, n_open=5)
    p = _plan(c, q, n_slice_edges=4)
    for qb, g in p.sliced_edges():
        assert c.q1[g] >= 0 and qb in (c.q0[g], c.q1[g])
        # the wire continues into a later two-qubit gate (internal edge)
        later = [h for h in range(g + 1, c.n_gates) if c.q1[h] >= 0 and qb in (c.q0[h], c.q1[h])]
        assert later


def test_workspace_covers_largest_intermediate():
    c, q = rqcgen.small_grid(4, 5, 12, seed=4, n_open=6)
    for dt, esz in ((tn.C64, 8), (tn.F16, 4)):
        i = _plan(c, q, dtype=dt, n_slice_edges=2).info()
        assert i["workspace_bytes"] >= esz << i["max_log2_elems"]


def test_plan_is_deterministic():
    c, q = rqcgen.small_grid(4, 5, 12, seed=4, n_open=6)
    a = _plan(c, q, n_slice_edges=3, trials=3, seed=9)
    b = _plan(c, q, n_slice_edges=3, trials=3, seed=9)
    assert a.sliced_edges() == b.sliced_edges() and a.steps() == b.steps()


def test_annealed_plan_does_not_depend_on_the_threads():
    # the annealing starts and chains run on threads of their own; the plan
    # they choose must be the same on every run (ties go to the lower start)
    c, q = rqcgen.small_grid(5, 6, 12, seed=2, n_open=8)
    kw = dict(n_slice_edges=-1, max_log2_elems=16, trials=4, seed=5, anneal_iters=3000)
    runs = [_plan(c, q, **kw) for _ in range(4)]
    ref = (runs[0].sliced_edges(), runs[0].steps(), runs[0].info()["flops_per_slice"])
    for p in runs[1:]:
        assert (p.sliced_edges(), p.steps(), p.info()["flops_per_slice"]) == ref


def test_rejects_bad_inputs():
    c, q = rqcgen.small_grid(3, 3, 4, seed=1, n_open=3)
    bad = rqcgen.Circuit(c.n_qubits, c.q0.copy(), c.q1.copy(), c.mats.copy())
    bad.q0[5] = 99
    with pytest.raises(tn.TnError) as e:
        _plan(bad, q)
    assert e.value.code == tn.TN_EINVAL
    q2 = rqcgen.Query(np.array([5, 2], dtype=np.int32), q.fixed_bits)
    with pytest.raises(tn.TnError):
        _plan(c, q2)  # not ascending
    with pytest.raises(tn.TnError):
        _plan(c, q, dtype=7)
    with pytest.raises(tn.TnError):
        _plan(c, q, n_slice_edges=1, slice_batch_log2=2)
    nan = rqcgen.Circuit(c.n_qubits, c.q0.copy(), c.q1.copy(), c.mats.copy())
    nan.mats[0, 0, 0] = np.nan
    with pytest.raises(tn.TnError):
        _plan(nan, q)


def test_workload_plans():
    # the 30-qubit workload: 8 sliced edges, 256 slices, 1024 amplitudes
    c, q = rqcgen.grid_30q()
    i = _plan(c, q, n_slice_edges=8, trials=4).info()
    assert i["n_slices"] == 256 and i["n_open"] == 10 and i["n_leaves"] == 172
    # the 53-qubit workload: sliced until each slice's largest tensor <= 2^30
    c, q = rqcgen.grid_53q()
    i = _plan(c, q, n_slice_edges=-1, max_log2_elems=30, trials=2).info()
    assert i["max_log2_elems"] <= 30 and i["n_open"] == 12


def test_plan_path_replayed_by_tn_oracle():
    # the planner's path and slicing, handed to the FP64 network oracle as
    # data, give the projector state vector's slices: the leaf sources and
    # step ids mean what the header says
    from oracle import tn as otn
    c, q = rqcgen.small_grid(3, 4, 8, seed=3, n_open=4)
    p = tn.Plan(c, q, dtype=tn.C64, n_slice_edges=2, torch_allocator=False)
    keys = [("g", g) if g >= 0 else ("q", qq) for g, qq in p.leaf_sources()]
    assert sorted(keys) == sorted(otn.leaf_keys(c))
    st = p.steps()
    assert [s["c"] for s in st] == list(range(len(keys), len(keys) + len(st)))
    steps = [(s["a"], s["b"]) for s in st]
    edges = p.sliced_edges()
    for sid in range(4):
        got = otn.contract(c, q, keys, steps, fixed=otn.slice_fixed(edges, sid))
        want = oracle.sliced_amplitudes(c, q, edges, [sid])
        assert np.max(np.abs(got - want)) <= 1e-13


def test_fp8_steps_are_marked_and_quantized():
    c, q = rqcgen.grid_30q()
    base = tn.Plan(c, q, dtype=tn.F16, n_slice_edges=8, trials=4, torch_allocator=False)
    p = tn.Plan(c, q, dtype=tn.F16, n_slice_edges=8, trials=4, torch_allocator=False,
                fp8_min_log2_flops=36)
    s0, s1 = base.steps(), p.steps()
    marked = [i for i, s in enumerate(s1) if s["storage"] & 8]
    assert marked
    for i in marked:
        s = s1[i]
        # only tensor-core steps with K >= 64 at or above the threshold
        assert s["kernel"] == 3 and s["log2_k"] >= 6
        assert s["log2_m"] + s["log2_n"] + s["log2_k"] + s["log2_batch"] + 3 >= 36
    for i, s in enumerate(s1):
        if i not in marked and s["kernel"] == 3 and s["log2_k"] >= 6:
            assert s["log2_m"] + s["log2_n"] + s["log2_k"] + s["log2_batch"] + 3 < 36
        assert (s["storage"] & 7) == s0[i]["storage"]
    # the E4M3 copies are extra traffic, the flops are unchanged
    assert p.info()["flops_per_slice"] == base.info()["flops_per_slice"]
    assert p.info()["bytes_per_slice"] > base.info()["bytes_per_slice"]
    c64 = tn.Plan(c, q, dtype=tn.C64, n_slice_edges=8, trials=4, torch_allocator=False, fp8_min_log2_flops=1)
    assert not any(s["storage"] & 8 for s in c64.steps())


@pytest.mark.parametrize("n_slice,cap,batch", [(2, 0, 0), (-1, 7, 0), (3, 0, 3)])
def test_annealed_path_is_valid_and_cheaper(n_slice, cap, batch):
    # simulated annealing over tree rotations (Sec. 3 path search): the
    # refined path and its slices still give the projector state vector's
    # slices (FP64 network oracle, path as data), within the same width,
    # for no more flops than the greedy path -- as the plan runs them (with
    # all slices in one batched pass, a step counts once per slice reaching it)
    from oracle import tn as otn
    c, q = rqcgen.small_grid(3, 4, 8, seed=3, n_open=4)
    kw = dict(dtype=tn.C64, n_slice_edges=n_slice, max_log2_elems=cap, torch_allocator=False,
              slice_batch_log2=batch)
    g = tn.Plan(c, q, **kw)
    a = tn.Plan(c, q, anneal_iters=20000, **kw)
    gi, ai = g.info(), a.info()
    total = lambda i: i["flops_per_slice"] * i["n_slices"] + i["flops_invariant"]
    assert total(ai) <= total(gi)
    if cap:
        assert ai["max_log2_elems"] <= cap
    else:
        assert ai["max_log2_elems"] <= gi["max_log2_elems"]
    keys = [("g", gg) if gg >= 0 else ("q", qq) for gg, qq in a.leaf_sources()]
    steps = [(s["a"], s["b"]) for s in a.steps()]
    edges = a.sliced_edges()
    full = 0
    for sid in range(ai["n_slices"]):
        got = otn.contract(c, q, keys, steps, fixed=otn.slice_fixed(edges, sid))
        assert np.max(np.abs(got - oracle.sliced_amplitudes(c, q, edges, [sid]))) <= 1e-13
        full = full + got
    assert np.max(np.abs(full - oracle.amplitudes(c, q))) <= 1e-13


def test_gather_rejects_bad_indices_before_touching_the_device():
    L = tn.lib()
    fake = ctypes.c_void_p(256)
    ia = (ctypes.c_int32 * 3)(0, 5, 1)
    ib = (ctypes.c_int32 * 3)(0, 0, 0)
    rc = L.tn_gemm_gather(tn.F16, fake, 4, fake, 2, fake, 3, 128, 8, 64, ia, ib, tn.GATHER_DIRECT, 0,
                          None, None, None)
    assert rc == tn.TN_EINVAL and "out of range" in L.tn_last_error().decode()
    ia2 = (ctypes.c_int32 * 3)(2, 1, 3)
    rc = L.tn_gemm_gather(tn.F16, fake, 4, fake, 2, fake, 3, 128, 8, 64, ia2, ib, tn.GATHER_PADDED, 0,
                          None, None, None)
    assert rc == tn.TN_EINVAL and "non-decreasing" in L.tn_last_error().decode()
    rc = L.tn_gemm_gather(tn.F16, fake, 4, fake, 2, fake, 3, 128, 8, 1 << 16, ia2, ib, tn.GATHER_DIRECT, 0,
                          None, None, None)
    assert rc == tn.TN_EUNSUPPORTED


def test_bundled_timings_for_the_cost_model():
    recs = tn.load_timings()
    if not recs:
        pytest.skip("no bundled timings")
    assert len(recs) >= 40000
    kinds = {r["kind"] for r in recs}
    assert kinds == {0, 1}
    assert all(r["ms"] > 0 for r in recs)
    x = tn.cost_features(recs[:1000])
    assert x.shape == (1000, tn.COST_NFEAT) and np.isfinite(x).all()


def test_sample_plan_builds_on_the_host():
    c, _ = rqcgen.small_grid(3, 4, 8, seed=3, n_open=4)
    rng = np.random.default_rng(0)
    s = rng.integers(0, 2, size=(10, 12))
    p = tn.Plan.from_samples(c, s, dtype=tn.C64, n_slice_edges=2, torch_allocator=False)
    assert p.info()["n_open"] == 4 and p.n_samples == 10
    with pytest.raises(tn.TnError):
        tn.Plan.from_samples(c, np.full((3, 12), 2), dtype=tn.C64, torch_allocator=False)


def test_sample_plan_cost_grows_slowly_with_the_sample_count():
    # tensors keep the output legs dense while they carry at most
    # log2(n_samples) of them, so 1024 bitstrings cost a few times one
    # bitstring, not 1024 times
    c, _ = rqcgen.grid_30q()
    rng = np.random.default_rng(1)
    flops = []
    for ns in (1, 1024):
        s = rng.integers(0, 2, size=(ns, 30))
        i = tn.Plan.from_samples(c, s, dtype=tn.F16, n_slice_edges=8, trials=4, torch_allocator=False).info()
        flops.append(i["flops_per_slice"] * i["n_slices"] + i["flops_invariant"])
    assert flops[1] < 16 * flops[0]
    # slices run together carry their own batch modes through the gathers
    i = tn.Plan.from_samples(c, np.zeros((4, 30)), dtype=tn.F16, n_slice_edges=8, slice_batch_log2=2,
                             torch_allocator=False).info()
    assert i["slice_batch_log2"] == 2 and i["n_open"] == 2


def test_recompute_plan_splits_open_legs():
    c, q = rqcgen.grid_30q()
    p = tn.Plan(c, q, dtype=tn.F16, n_slice_edges=8, trials=4, slice_batch_log2=8, recompute_log2=2,
                torch_allocator=False)
    i = p.info()
    assert i["n_recompute_edges"] == 2 and i["n_slice_edges"] == 10 and i["n_slices"] == 1 << 10
    assert {qq for qq, _ in p.sliced_edges()[-2:]} <= set(q.open_qubits)
    c2, q2 = rqcgen.small_grid(3, 4, 8, seed=3, n_open=2)
    with pytest.raises(tn.TnError, match="open output legs"):
        tn.Plan(c2, q2, dtype=tn.F16, recompute_log2=3, torch_allocator=False)   # 2 open legs
    with pytest.raises(tn.TnError):
        tn.Plan.from_samples(c, np.zeros((4, 30)), dtype=tn.F16, recompute_log2=1, torch_allocator=False)


def test_cost_features_mark_cta_pair_tiles():
    # slot 25 of a tensor-core GEMM record flags CTA-pair tiles, only where
    # the shape runs on pairs (M >= 256, N >= 128 complex, K >= 32)
    base = dict(kind=0, lm=16, ln=12, lk=10, lb=0, dtype=tn.F16, kernel=3)
    recs = [dict(base, tile=0), dict(base, tile=0x100), dict(base, lm=7, tile=0x100),
            dict(base, ln=5, tile=0x100), dict(base, lk=4, tile=0x100), dict(base, tile=0x141)]
    x = tn.cost_features(recs)
    assert x[:, 25].tolist() == [0.0, 1.0, 0.0, 0.0, 0.0, 1.0]
    # the pair bit does not change the other features of the record
    assert np.array_equal(np.delete(x[0], 25), np.delete(x[1], 25))


def test_workspace_budget_picks_the_largest_fitting_slice_batch():
    # tn_plan_opts.workspace_budget: one path search, then the largest slice
    # batch whose workspace fits the budget (else no batching)
    items = rqcgen.uneven_batch()
    for i in (2, 14, 17):
        c, q = items[i]
        budget = 1 << 30
        p = tn.plan_within_budget(c, q, dtype=tn.F16, torch_allocator=False, workspace_budget=budget)
        info = p.info()
        b, s = info["slice_batch_log2"], info["n_slice_edges"]
        assert info["workspace_bytes"] <= budget or b == 0
        if b < min(s, 16):
            nxt = _plan(c, q, dtype=tn.F16, n_slice_edges=-1, max_log2_elems=24, trials=4, slice_batch_log2=b + 1)
            assert nxt.info()["workspace_bytes"] > budget
            assert nxt.sliced_edges() == p.sliced_edges()


def test_cost_targets_are_log2_microseconds():
    recs = [{"ms": 1.0}, {"ms": 0.25}, {"ms": 1e-9}]
    np.testing.assert_allclose(tn.cost_targets(recs), [np.log2(1e3), np.log2(250.0), np.log2(1e-3)], rtol=1e-6)


def test_allocator_callback_returns_null_when_torch_cannot_allocate():
    # an exception may not leave the ctypes callback (the library would get an
    # undefined pointer); without a GPU torch.empty(device="cuda") raises, and
    # the callback must answer NULL so that the library reports TN_ENOMEM
    import torch
    if torch.cuda.is_available():
        pytest.skip("needs a process without a GPU")
    a = tn._TorchAllocator()
    assert a.alloc(1 << 20, None) is None
    a.free(None, None)
    assert not a._live


@pytest.mark.parametrize("kind", ["sliced", "annealed", "recompute", "samples"])
def test_plan_flops_are_the_steps_8mnk(kind):
    # the TFLOP/s figures divide the plan's flops by time: they must be the
    # method's own work, 8 M N K real flops per complex GEMM step (Sec. 3.3,
    # Eq. 6), each step counted once per pass of 2^b slices, or once per
    # call for the steps that no looped sliced edge reaches
    c, q = rqcgen.small_grid(4, 5, 12, seed=4, n_open=8)
    if kind == "sliced":
        p = _plan(c, q, n_slice_edges=4, slice_batch_log2=2)
    elif kind == "annealed":
        c, q = rqcgen.small_grid(5, 6, 12, seed=2, n_open=8)
        p = _plan(c, q, n_slice_edges=-1, max_log2_elems=16, anneal_iters=3000, slice_batch_log2=1)
    elif kind == "recompute":
        p = _plan(c, q, n_slice_edges=2, recompute_log2=2, slice_batch_log2=1)
    else:
        bits = np.random.default_rng(1).integers(0, 2, size=(100, c.n_qubits)).astype(np.uint8)
        p = tn.Plan.from_samples(c, bits, dtype=tn.F16, n_slice_edges=2, slice_batch_log2=1,
                                 torch_allocator=False)
    i = p.info()
    passes = i["n_slices"] >> i["slice_batch_log2"]
    total = 0.0
    for s in p.steps():
        f = 8.0 * 2.0 ** (s["log2_m"] + s["log2_n"] + s["log2_k"] + s["log2_batch"])
        total += f if s["slice_invariant"] else f * passes
    assert total == i["flops_per_slice"] * i["n_slices"] + i["flops_invariant"]
    assert any(not s["slice_invariant"] for s in p.steps()) or i["n_slices"] == 1


def test_no_fallback_when_the_library_cannot_load(monkeypatch, tmp_path):
    # there is no CPU path behind the binding: a library that cannot be
    # built or loaded makes every call raise
    bad = tmp_path / "libtn.so"
    bad.write_bytes(b"not a shared library")
    monkeypatch.setattr(tn, "_lib", None)
    monkeypatch.setattr(tn._build_mod, "build", lambda force=False: str(bad))
    c, q = rqcgen.small_grid(3, 3, 4, seed=1, n_open=3)
    with pytest.raises(OSError):
        tn.Plan(c, q, torch_allocator=False)

    def no_toolkit(force=False):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    monkeypatch.setattr(tn._build_mod, "build", no_toolkit)
    with pytest.raises(RuntimeError, match="nvcc not found"):
        tn.lib()
