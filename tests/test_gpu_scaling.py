"""Pins of the per-tensor power-of-two scaling of complex-half plans and of
the slice decoding, through the C ABI.

The paper computes in complex-half (Sec. 3.3) without saying how values are
kept inside FP16's range; this library scales every stored tensor by an
exact 2^e chosen on the device and divides it out in the FP64 slice sum.
These tests check that the scaling is exact, that it lands where it claims,
and that without it the 30-qubit workload misses the accuracy budget.  The
slice decoding (Sec. 3.1: bit j of the slice id is the value of sliced edge
j, LSB first) is checked bit for bit against an indexing of the leaf written
here in numpy."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
import rqcgen  # noqa: E402
import paper_2407_00769_gb300 as tn  # noqa: E402

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")

FP16_MIN_NORMAL = 2.0 ** -14


def _golden_30q():
    vals = []
    for line in open(os.path.join(GOLD, "grid5x6_14c_amps.txt")):
        if line.startswith("#") or not line.strip():
            continue
        _, re_, im_ = line.split()
        vals.append(complex(float(re_), float(im_)))
    return np.array(vals)


# ---------------------------------------------------------------- exactness --

def _scaled_circuit(c, gate, m):
    mats = c.mats.copy()
    mats[gate] = np.ldexp(mats[gate].real, m) + 1j * np.ldexp(mats[gate].imag, m)
    return rqcgen.Circuit(c.n_qubits, c.q0, c.q1, mats)


@pytest.mark.parametrize("dtype", [tn.F16, tn.BF16, tn.C64])
@pytest.mark.parametrize("m", [-7, 5])
def test_scaled_gate_scales_result_exactly(dtype, m):
    # The network is linear in every gate.  Multiplying one gate by 2^m
    # multiplies every tensor downstream of it by 2^m; the device's exponents
    # shift by -m, the stored complex-half values stay bit-identical, and the
    # FP64 slice sum's ldexp undoes the shift exactly.  So the amplitudes must
    # be exactly 2^m times the unscaled ones: the scale-then-unscale round
    # trip of the whole path is exact.
    c, q = rqcgen.small_grid(4, 4, 10, seed=11, n_open=6)
    g2 = int(np.nonzero(c.q1 >= 0)[0][3])
    kw = dict(dtype=dtype, n_slice_edges=3, small_log2=6, slice_batch_log2=1)
    base = tn.Plan(c, q, **kw).contract().cpu().numpy()
    scaled = tn.Plan(_scaled_circuit(c, g2, m), q, **kw).contract().cpu().numpy()
    want = np.ldexp(base.real, m) + 1j * np.ldexp(base.imag, m)
    assert np.array_equal(scaled.view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("dtype,kernel", [(tn.F16, 2), (tn.F16, 3), (tn.F16, tn.GEMM_TC_PAIR),
                                          (tn.BF16, 2), (tn.BF16, 3)])
@pytest.mark.parametrize("e", [-6, -1, 3, 9])
def test_epilogue_power_of_two_is_exact(dtype, kernel, e):
    # The epilogue multiplies the FP32 accumulator by 2^e before rounding.
    # Rounding commutes with a power-of-two factor while both values are
    # normal, so C(e) must equal 2^e C(0) bit for bit on every element whose
    # values are normal in both.
    M, N, K = 512, 128, 64
    g = torch.Generator().manual_seed(7 + e)
    tdt = torch.float16 if dtype == tn.F16 else torch.bfloat16
    A = (torch.randn(M, K, 2, generator=g) * 0.25).to(tdt).cuda()
    B = (torch.randn(K, N, 2, generator=g) * 0.25).to(tdt).cuda()
    C0 = torch.empty(M, N, 2, dtype=tdt, device="cuda")
    Ce = torch.empty_like(C0)
    tn.gemm(dtype, A, B, C0, M, N, K, scale_exp=0, kernel=kernel)
    tn.gemm(dtype, A, B, Ce, M, N, K, scale_exp=e, kernel=kernel)
    c0 = C0.float().cpu().numpy().astype(np.float64)
    ce = Ce.float().cpu().numpy().astype(np.float64)
    lo = FP16_MIN_NORMAL if dtype == tn.F16 else 2.0 ** -126
    ok = (np.abs(c0) >= lo) & (np.abs(np.ldexp(c0, e)) >= lo)
    assert ok.mean() > 0.95
    assert np.array_equal(ce[ok], np.ldexp(c0[ok], e))


# ---------------------------------------------------------- exponent window --

def _check_window(p):
    n_half, n_head = 0, 0
    for i, st in enumerate(p.steps()):
        if not (st["storage"] & 4):          # output kept complex64: e = 0
            continue
        E, mx = p.step_scale(i)
        n_half += 1
        # the bound caps the stored maximum at 2^14; calibration lifts a step
        # whose maximum is below 2^12 into (2^11, 2^12]
        assert 2.0 ** 11 < mx <= 2.0 ** 14, (i, mx, st)
        if st["scale_headroom"] > 0:
            n_head += 1
            assert mx <= 2.0 ** 12, (i, mx, st)
    return n_half, n_head


@pytest.mark.parametrize("dtype", [tn.F16, tn.BF16])
def test_exponent_window_small_circuit(dtype):
    # one pass covers every slice (slice_batch_log2 = n_slice_edges), so the
    # pass read back is the calibration pass the window is stated for
    # small_log2 = 4 stores every tensor above 16 elements in complex-half,
    # many more roundings than the default rule (2^16); the accuracy check
    # here is the FP16 budget, scaled for BF16 by the ratio of unit roundoffs
    # (2^-8 / 2^-11 = 8)
    c, q = rqcgen.small_grid(4, 5, 12, seed=8, n_open=6)
    p = tn.Plan(c, q, dtype=dtype, n_slice_edges=3, slice_batch_log2=3, small_log2=4)
    got = p.contract().cpu().numpy()
    assert oracle.rel_l2(got, oracle.amplitudes(c, q)) <= (5e-3 if dtype == tn.F16 else 8 * 5e-3)
    n_half, n_head = _check_window(p)
    assert n_half >= 10 and n_head >= 1


def test_exponent_window_30q():
    # the benchmark's workload: FP16, 256 slices in one pass
    c, q = rqcgen.grid_30q()
    p = tn.Plan(c, q, dtype=tn.F16, n_slice_edges=8, trials=4, slice_batch_log2=8)
    got = p.contract().cpu().numpy()
    assert oracle.rel_l2(got, _golden_30q()) <= 5e-3
    n_half, n_head = _check_window(p)
    print(f"grid30 f16: {n_half} complex-half step outputs in the window, {n_head} with headroom")
    assert n_half >= 10


# ---------------------------------------------------------- scaling disabled --

def test_scaling_off_misses_the_budget_30q():
    # Negative pin: the same FP16 job with every exponent 0.  One slice's
    # share of an amplitude is about 2^-15 / 16 (2^30 amplitudes of mean
    # |amp|^2 = 2^-30, 256 slices adding with random phases), so the final
    # tensor of a pass holds values near 2^-19: inside FP16's subnormal range
    # (below 2^-14), where the spacing 2^-24 leaves about 5 significant bits.
    # The scaled path keeps the same values near 2^12.
    want = _golden_30q()
    c, q = rqcgen.grid_30q()
    kw = dict(dtype=tn.F16, n_slice_edges=8, trials=4, slice_batch_log2=8)
    on = tn.Plan(c, q, **kw)
    e_on = oracle.rel_l2(on.contract().cpu().numpy(), want)
    off = tn.Plan(c, q, no_scaling=True, **kw)
    try:
        got, _ = off.contract(report=True)
    except tn.TnError as ex:
        # a value above FP16's range is the other way the unscaled path fails
        assert ex.code == tn.TN_EUNSUPPORTED
        print(f"grid30 f16 without scaling: overflow ({ex}); with scaling rel_l2={e_on:.3e}")
        return
    e_off = oracle.rel_l2(got.cpu().numpy(), want)
    last = max(i for i, st in enumerate(off.steps()) if st["storage"] & 4)
    E, mx = off.step_scale(last)
    print(f"grid30 f16: rel_l2 {e_on:.3e} scaled, {e_off:.3e} without scaling "
          f"(last complex-half output max {mx:.3e}, exponent {E})")
    assert e_on <= 5e-3
    assert E == 0
    assert mx < FP16_MIN_NORMAL          # the whole final tensor is subnormal
    assert not e_off <= 5e-3             # the budget is missed (or NaN)


def test_no_scaling_option_rejects_fp8():
    c, q = rqcgen.small_grid(3, 3, 6, seed=2, n_open=3)
    with pytest.raises(tn.TnError):
        tn.Plan(c, q, dtype=tn.F16, no_scaling=True, fp8_min_log2_flops=30)


# ------------------------------------------------------------- slice decode --

def _expected_leaf(full_legs, full, sliced, batch_log2, slice_id, kept_legs):
    """Pick the sub-tensor of a full leaf that a slice fixes: sliced edge j
    takes bit j of the slice id (LSB first); edges j < batch_log2 run as
    batch modes and stay legs.  Then lay the kept legs out in kept_legs order
    and round to complex64."""
    fixed = {}
    for j, edge in enumerate(sliced):
        if j >= batch_log2:
            fixed[edge] = (slice_id >> j) & 1
    index = tuple(fixed[leg] if leg in fixed else slice(None) for leg in full_legs)
    sub = full[index]
    rest = [leg for leg in full_legs if leg not in fixed]
    assert sorted(rest) == sorted(kept_legs)
    sub = np.transpose(sub, [rest.index(leg) for leg in kept_legs]) if rest else sub
    return np.ascontiguousarray(sub).astype(np.complex64)


@pytest.mark.parametrize("n_edges,batch", [(3, 0), (5, 0), (5, 2), (4, 4)])
def test_slice_decoding_bit_exact(n_edges, batch):
    c, q = rqcgen.small_grid(4, 4, 10, seed=7, n_open=6)
    p = tn.Plan(c, q, dtype=tn.F16, n_slice_edges=n_edges, trials=2, slice_batch_log2=batch)
    sliced = p.sliced_edges()
    assert len(sliced) == n_edges
    n_leaves = p.info()["n_leaves"]
    touched = 0
    for sid in range(0, 1 << n_edges, 1 << batch):
        for i in range(n_leaves):
            full_legs, full = p.leaf_tensor(i)
            kept_legs, got = p.decode_leaf(sid, i)
            want = _expected_leaf(full_legs, full, sliced, batch, sid, kept_legs)
            assert got.shape == want.shape
            assert np.array_equal(got.reshape(-1).view(np.uint32), want.reshape(-1).view(np.uint32)), (sid, i)
            touched += any(leg in sliced for leg in full_legs)
    assert touched > 0
    # a pass must start on a batch boundary
    if batch > 0:
        with pytest.raises(tn.TnError):
            p.decode_leaf(1, 0)
