"""Single-kernel parity through the C ABI: bit-exact permutations, complex
GEMMs (complex64 SIMT, complex-half rows, tcgen05 tensor cores) against FP64
products of the same (rounded) inputs, and the paper's worked complex-half
example (Sec. 3.3) through the tensor-core path."""
import itertools
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2407_00769_gb300 as tn  # noqa: E402

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# ------------------------------------------------------------------ permute
@pytest.mark.parametrize("elem", [4, 8])
def test_permute_all_small_ranks(elem):
    dt = np.int32 if elem == 4 else np.int64
    for r in range(0, 6):
        x = np.arange(1 << r, dtype=dt) * 7 + 3
        xd = dev(x)
        for perm in itertools.permutations(range(r)):
            out = tn.permute(xd, list(perm), elem_bytes=elem)
            want = np.transpose(x.reshape([2] * r), perm).reshape(-1) if r else x
            assert np.array_equal(out.cpu().numpy(), want), (r, perm)


@pytest.mark.parametrize("r", [6, 9, 11, 12, 16, 20])
def test_permute_random(r):
    rng = np.random.default_rng(r)
    for elem, dt in ((4, np.int32), (8, np.int64)):
        x = rng.integers(-2**31, 2**31 - 1, size=1 << r).astype(dt)
        xd = dev(x)
        for _ in range(4):
            perm = list(rng.permutation(r))
            out = tn.permute(xd, perm, elem_bytes=elem)
            want = np.transpose(x.reshape([2] * r), perm).reshape(-1)
            assert np.array_equal(out.cpu().numpy(), want), perm


def test_permute_large_reversal():
    r = 24
    x = torch.arange(1 << r, dtype=torch.int32, device="cuda")
    perm = list(range(r))[::-1]
    out = tn.permute(x, perm).cpu().numpy()
    idx = np.arange(1 << r, dtype=np.int64)
    rev = np.zeros_like(idx)
    for b in range(r):
        rev |= ((idx >> b) & 1) << (r - 1 - b)
    assert np.array_equal(out, rev.astype(np.int32))


# --------------------------------------------------------------------- gemm
def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def to_c64(z):
    return z.astype(np.complex64)


def half_pairs(z, np_dtype=np.float16):
    r = np.empty(z.shape + (2,), dtype=np_dtype)
    r[..., 0] = z.real
    r[..., 1] = z.imag
    return r


def from_pairs(a):
    a = a.astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


def bf16_round(z):
    t = torch.from_numpy(np.stack([z.real, z.imag], -1).astype(np.float32)).to(torch.bfloat16)
    return t


def ref_gemm(a, b):
    return np.matmul(a.astype(np.complex128), b.astype(np.complex128))


def bound(a, b, K):
    return np.matmul(np.abs(a), np.abs(b))


C64_SHAPES = [(1, 1, 1), (3, 2, 4), (128, 4, 4), (1000, 8, 16), (4096, 2, 1), (64, 64, 16),
              (256, 128, 64), (128, 16, 256), (2, 256, 2),
              # 128 x 128 tiles of the tiled kernel (M N >= 2^18)
              (1024, 256, 64), (512, 512, 16), (2048, 128, 1024)]


@pytest.mark.parametrize("M,N,K", C64_SHAPES)
@pytest.mark.parametrize("batch", [1, 3])
def test_gemm_c64(M, N, K, batch):
    M = 1 << int(np.ceil(np.log2(M)))
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    a = to_c64(crandn(rng, batch, M, K))
    b = to_c64(crandn(rng, batch, K, N))
    c = torch.zeros(batch, M, N, dtype=torch.complex64, device="cuda")
    for kernel in (-1, 0, 1):
        if kernel == 1 and not (M >= 64 and N >= 64 and K >= 16):
            continue
        tn.gemm(tn.C64, dev(a), dev(b), c, M, N, K, batch=batch, batch_a=True, batch_b=True,
                kernel=kernel)
        got = c.cpu().numpy()
        want = ref_gemm(a, b)
        err = np.abs(got - want)
        assert np.all(err <= 1e-6 * bound(a, b, K) * max(1, np.sqrt(K)) + 1e-30), kernel


# complex64 on the tensor cores (tn_gemm kernel 9): each FP32 operand split
# into a TF32 part and its remainder, three kind::tf32 MMAs per K slice.
# Per product the dropped and truncated parts are below ~2^-19 of |a||b|, so
# the error bound is the complex64 path's with a few units of FP32 rounding,
# and rel-L2 stays within the complex64 budget (1e-5).
@pytest.mark.parametrize("M,N,K,batch", [(128, 8, 8, 1), (256, 64, 64, 2), (1024, 256, 512, 1),
                                         (64, 16, 16, 3), (4096, 128, 32, 1), (512, 512, 2048, 1)])
def test_gemm_c64_tensor_cores(M, N, K, batch):
    rng = np.random.default_rng(M * 11 + N * 5 + K)
    a = to_c64(crandn(rng, batch, M, K))
    b = to_c64(crandn(rng, batch, K, N))
    c = torch.zeros(batch, M, N, dtype=torch.complex64, device="cuda")
    mx = torch.zeros(1, dtype=torch.float32, device="cuda")
    tn.gemm(tn.C64, dev(a), dev(b), c, M, N, K, batch=batch, batch_a=True, batch_b=True, kernel=9, out_max=mx)
    got = c.cpu().numpy().astype(np.complex128)
    want = ref_gemm(a, b)
    err = np.abs(got - want)
    assert np.all(err <= 4e-6 * bound(a, b, K) * max(1, np.sqrt(K)) + 1e-30)
    assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)
    # the recorded maximum is that of the stored components
    assert mx.item() == pytest.approx(float(np.max(np.abs(np.stack([got.real, got.imag])))), rel=1e-6)


def test_gemm_c64_tensor_cores_broadcast_b():
    rng = np.random.default_rng(9)
    M, N, K, batch = 256, 32, 64, 4
    a = to_c64(crandn(rng, batch, M, K))
    b = to_c64(crandn(rng, K, N))
    c = torch.zeros(batch, M, N, dtype=torch.complex64, device="cuda")
    tn.gemm(tn.C64, dev(a), dev(b), c, M, N, K, batch=batch, batch_a=True, batch_b=False, kernel=9)
    want = ref_gemm(a, np.broadcast_to(b, (batch, K, N)))
    got = c.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)


def test_gemm_c64_broadcast_b():
    rng = np.random.default_rng(5)
    M, N, K, batch = 256, 8, 8, 4
    a = to_c64(crandn(rng, batch, M, K))
    b = to_c64(crandn(rng, K, N))
    c = torch.zeros(batch, M, N, dtype=torch.complex64, device="cuda")
    tn.gemm(tn.C64, dev(a), dev(b), c, M, N, K, batch=batch, batch_a=True, batch_b=False)
    assert np.allclose(c.cpu().numpy(), ref_gemm(a, b[None]), rtol=1e-5, atol=1e-5)


LP_SHAPES = [(1, 1, 8), (2, 4, 8), (128, 8, 8), (256, 16, 16), (4096, 4, 32), (1024, 128, 64),
             (512, 256, 512), (256, 1, 1024), (64, 64, 8), (8192, 2, 8), (256, 512, 64)]


def _lp_case(dtype, M, N, K, batch, kernel, ba=True, bb=True, seed=0):
    rng = np.random.default_rng(seed + M * 13 + N * 5 + K)
    a = crandn(rng, batch if ba else 1, M, K)
    b = crandn(rng, batch if bb else 1, K, N) / np.sqrt(K)
    if dtype == tn.F16:
        ah, bh = half_pairs(a), half_pairs(b)
        ad, bd = dev(ah), dev(bh)
        ar, br = from_pairs(ah), from_pairs(bh)
        unit = 2.0 ** -11
    else:
        ad, bd = bf16_round(a).cuda(), bf16_round(b).cuda()
        ar = ad.float().cpu().numpy().astype(np.float64)
        ar = ar[..., 0] + 1j * ar[..., 1]
        br = bd.float().cpu().numpy().astype(np.float64)
        br = br[..., 0] + 1j * br[..., 1]
        unit = 2.0 ** -8
    c = torch.zeros(batch, M, N, 2, dtype=torch.float16 if dtype == tn.F16 else torch.bfloat16,
                    device="cuda")
    mx = torch.zeros(1, dtype=torch.float32, device="cuda")
    tn.gemm(dtype, ad, bd, c, M, N, K, batch=batch, batch_a=ba, batch_b=bb, scale_exp=3,
            kernel=kernel, out_max=mx)
    got = c.float().cpu().numpy().astype(np.float64)
    got = got[..., 0] + 1j * got[..., 1]
    want = ref_gemm(np.broadcast_to(ar, (batch, M, K)), np.broadcast_to(br, (batch, K, N))) * 8.0
    mag = 8.0 * np.matmul(np.abs(np.broadcast_to(ar, (batch, M, K))), np.abs(np.broadcast_to(br, (batch, K, N))))
    tol = 2 * unit * np.abs(want) + 1e-6 * mag + 1e-30
    assert np.all(np.abs(got - want) <= tol), (np.max(np.abs(got - want) / (np.abs(want) + 1e-9)))
    gmax = max(np.abs(got.real).max(), np.abs(got.imag).max())
    assert abs(mx.item() - gmax) <= 1e-6 * gmax


@pytest.mark.parametrize("M,N,K", LP_SHAPES)
def test_gemm_f16_tensor_cores(M, N, K):
    _lp_case(tn.F16, M, N, K, 1, 3)


@pytest.mark.parametrize("M,N,K", [(128, 8, 8), (1024, 128, 64), (512, 256, 512)])
def test_gemm_bf16_tensor_cores(M, N, K):
    _lp_case(tn.BF16, M, N, K, 1, 3)


@pytest.mark.parametrize("ba,bb", [(True, True), (True, False), (False, True)])
def test_gemm_f16_tensor_cores_batched(ba, bb):
    _lp_case(tn.F16, 256, 16, 32, 3, 3, ba, bb)


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (128, 4, 2), (300, 16, 4), (1024, 64, 1), (256, 8, 64),
                                   (128, 128, 512), (1 << 16, 4, 4), (16, 1 << 20, 4)])
def test_gemm_f16_rows(M, N, K):
    # (128, 128, 512): few row blocks, fewer columns per thread to fill the
    # GPU, FP64 partials (K > 256); (2^16, 4, 4): row blocks looped over by a
    # capped grid; (16, 2^20, 4): 65536 column chunks, more than a grid holds
    M = 1 << int(np.ceil(np.log2(M)))
    _lp_case(tn.F16, M, N, K, 1 if N > 4096 else 2, 2)


# CTA pairs (cluster of 2, one M = 256 tcgen05.mma over both SMs): one tile,
# several m and n tiles, more pair tiles than the GPU holds pairs (each pair
# walks several tiles through both accumulator buffers), K rings that wrap,
# and shapes the pair kernel does not take (run by the 1-CTA kernel)
PAIR_SHAPES = [(256, 128, 32), (512, 256, 512), (1024, 128, 64), (32768, 128, 64), (4096, 256, 2048),
               (128, 128, 64), (256, 64, 64), (256, 128, 16)]


@pytest.mark.parametrize("M,N,K", PAIR_SHAPES)
def test_gemm_f16_tensor_cores_cta_pairs(M, N, K):
    _lp_case(tn.F16, M, N, K, 1, tn.GEMM_TC_PAIR)


@pytest.mark.parametrize("ba,bb", [(True, True), (True, False), (False, True)])
def test_gemm_tensor_cores_cta_pairs_batched(ba, bb):
    _lp_case(tn.F16, 512, 128, 64, 3, tn.GEMM_TC_PAIR, ba, bb)
    _lp_case(tn.BF16, 256, 256, 128, 2, tn.GEMM_TC_PAIR, ba, bb)


@pytest.mark.parametrize("M,N,K", [(256, 128, 32), (1024, 256, 512), (128, 64, 64), (4096, 128, 2048)])
def test_gemm_tensor_cores_half_k_chunks(M, N, K):
    # 64-byte K chunks (32 FP16 per row, 64-byte swizzle, twice the stages)
    _lp_case(tn.F16, M, N, K, 1, tn.GEMM_TC_HALF_K)
    _lp_case(tn.BF16, M, N, K, 2, tn.GEMM_TC_HALF_K)


# B'-resident kernel (each CTA keeps its B' slice in shared memory across its
# tiles; short K): against the reference within the rounding bound, and bit
# for bit against the 1-CTA kernel (same MMAs, same epilogue).  Shapes: one
# tile, N tiles that do / do not divide the grid (walkers whose slice changes),
# M below 128 (a partial tile), K = 8 .. 64 (32-, 64- and 128-byte K chunks), a K
# whose B' slice no longer fits (run by the 1-CTA kernel), many tiles per CTA.
BRES_SHAPES = [(128, 16, 8), (1024, 128, 16), (2048, 256, 32), (4096, 512, 64), (64, 64, 64),
               (65536, 32, 64), (1 << 17, 128, 16), (512, 1024, 8), (1024, 128, 256), (256, 4096, 64)]


def _gemm_bits(dtype, M, N, K, batch, ba, bb, kernel, seed=3):
    g = torch.Generator(device="cuda").manual_seed(seed + M + N + K)
    tdt = torch.float16 if dtype == tn.F16 else torch.bfloat16
    a = (torch.randn(batch if ba else 1, M, K, 2, generator=g, device="cuda") * 0.5).to(tdt)
    b = (torch.randn(batch if bb else 1, K, N, 2, generator=g, device="cuda") / K ** 0.5).to(tdt)
    c = torch.zeros(batch, M, N, 2, dtype=tdt, device="cuda")
    tn.gemm(dtype, a, b, c, M, N, K, batch=batch, batch_a=ba, batch_b=bb, scale_exp=2, kernel=kernel)
    return c.view(torch.int16).cpu().numpy()


@pytest.mark.parametrize("kernel", [tn.GEMM_TC_BRES, tn.GEMM_TC_BRES_STORE])
@pytest.mark.parametrize("M,N,K", BRES_SHAPES)
def test_gemm_tensor_cores_b_resident(M, N, K, kernel):
    # (GEMM_TC_BRES_STORE: C staged in shared memory and written by TMA
    # stores where N >= 32; the narrower shapes run as GEMM_TC_BRES)
    _lp_case(tn.F16, M, N, K, 1, kernel)
    assert np.array_equal(_gemm_bits(tn.F16, M, N, K, 1, True, True, kernel),
                          _gemm_bits(tn.F16, M, N, K, 1, True, True, 3))


@pytest.mark.parametrize("ba,bb", [(True, True), (True, False), (False, True)])
def test_gemm_tensor_cores_b_resident_batched(ba, bb):
    # a batched B changes each walker's slice with the batch entry
    _lp_case(tn.F16, 1024, 128, 32, 3, tn.GEMM_TC_BRES, ba, bb)
    _lp_case(tn.BF16, 512, 256, 64, 4, tn.GEMM_TC_BRES, ba, bb)
    _lp_case(tn.F16, 1024, 128, 32, 3, tn.GEMM_TC_BRES_STORE, ba, bb)
    for dt in (tn.F16, tn.BF16):
        for kern in (tn.GEMM_TC_BRES, tn.GEMM_TC_BRES_STORE):
            assert np.array_equal(_gemm_bits(dt, 2048, 64, 16, 5, ba, bb, kern),
                                  _gemm_bits(dt, 2048, 64, 16, 5, ba, bb, 3))


# Staged-store epilogue (each warp's rounded results through shared memory,
# whole 32-byte sectors per store): the same values as the row-per-thread
# stores, bit for bit, on tiles of 16-256 real columns, a partial M tile,
# batches and both half types; N = 4 (2N < 16) runs the row-per-thread path.
STAGED_SHAPES = [(128, 8, 8), (1024, 16, 16), (256, 32, 64), (4096, 64, 32), (64, 128, 128),
                 (1 << 14, 256, 16), (2048, 512, 256), (512, 4, 64)]


@pytest.mark.parametrize("M,N,K", STAGED_SHAPES)
def test_gemm_tensor_cores_staged_stores(M, N, K):
    _lp_case(tn.F16, M, N, K, 1, tn.GEMM_TC_STAGED)
    for dt in (tn.F16, tn.BF16):
        assert np.array_equal(_gemm_bits(dt, M, N, K, 1, True, True, tn.GEMM_TC_STAGED),
                              _gemm_bits(dt, M, N, K, 1, True, True, 3))
    assert np.array_equal(_gemm_bits(tn.F16, M, N, K, 3, True, False, tn.GEMM_TC_STAGED),
                          _gemm_bits(tn.F16, M, N, K, 3, True, False, 3))


def test_gemm_tensor_cores_cta_pairs_long_k():
    # K = 2^16 complex: split into K parts (FP32 partials, FP64 reduction)
    M, N, K = 256, 128, 1 << 16
    g = torch.Generator(device="cuda").manual_seed(5)
    a = torch.randn(1, M, K, 2, generator=g, device="cuda").half()
    b = (torch.randn(1, K, N, 2, generator=g, device="cuda") / K ** 0.5).half()
    c = torch.zeros(1, M, N, 2, dtype=torch.float16, device="cuda")
    tn.gemm(tn.F16, a, b, c, M, N, K, scale_exp=0, kernel=tn.GEMM_TC_PAIR)
    want = torch.matmul(torch.view_as_complex(a.double())[0], torch.view_as_complex(b.double())[0])
    got = torch.view_as_complex(c.double())[0]
    rel = (torch.linalg.norm(got - want) / torch.linalg.norm(want)).item()
    assert rel < 3e-4, rel


def _read_example():
    vals = {}
    for line in open(os.path.join(GOLD, "complex_half_example.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = [float(x) for x in v.split()]
    return vals


@pytest.mark.parametrize("kernel", [2, 3])
def test_paper_worked_example(kernel):
    # a1a2,b1 -> a1b1 with A = [(1+2i), (3+4i)], B = [(5+6i)]: the paper's
    # integer example, exact in FP16; embedded in a K = 8 step (zeros) so the
    # tensor-core path (K >= 8) runs it too.
    g = _read_example()
    M, N, K = 2, 1, 8
    A = np.zeros((M, K, 2), dtype=np.float16)
    A[0, 0] = g["A_complex"][0:2]
    A[1, 0] = g["A_complex"][2:4]
    B = np.zeros((K, N, 2), dtype=np.float16)
    B[0, 0] = g["B_complex"]
    C = torch.zeros(M, N, 2, dtype=torch.float16, device="cuda")
    tn.gemm(tn.F16, dev(A), dev(B), C, M, N, K, scale_exp=0, kernel=kernel)
    assert C.float().cpu().numpy().reshape(-1).tolist() == g["C_complex"]


def test_bounded_wait_times_out_and_context_survives():
    # the tensor-core GEMM's producer is told to issue nothing: the MMA
    # warp's mbarrier wait must give up (~2 s), report, free TMEM, return
    L = tn.lib()
    rc = L.tn_selftest_wait_timeout(torch.cuda.current_stream().cuda_stream)
    assert rc == tn.TN_ETIMEOUT, L.tn_last_error()
    # the context is still usable: a normal tensor-core GEMM is correct
    _lp_case(tn.F16, 256, 16, 32, 1, 3)


def test_bounded_wait_times_out_on_cta_pairs_and_context_survives():
    # the same on the CTA-pair kernel: both CTAs give up, meet at the
    # teardown barrier, free TMEM and return; then pairs compute correctly
    L = tn.lib()
    rc = L.tn_selftest_wait_timeout_pair(torch.cuda.current_stream().cuda_stream)
    assert rc == tn.TN_ETIMEOUT, L.tn_last_error()
    _lp_case(tn.F16, 512, 128, 64, 1, tn.GEMM_TC_PAIR)


@pytest.mark.parametrize("M,N,K", [(128, 32, 1 << 22), (1024, 32, 1 << 18), (128, 256, 1 << 16),
                                   (65536, 16, 1 << 12)])
def test_gemm_f16_tensor_cores_long_k(M, N, K):
    # Long contractions (the last steps of a sliced network reach K = 2^23):
    # the relative L2 error must stay at the level of the FP16 output rounding
    # (about 2e-4 for Gaussian data) whatever K is.  Reference: complex128
    # product of the same FP16-rounded operands, on the device.
    g = torch.Generator(device="cuda").manual_seed(K + M + N)
    a = torch.randn(1, M, K, 2, generator=g, device="cuda").half()
    b = (torch.randn(1, K, N, 2, generator=g, device="cuda") / K ** 0.5).half()
    c = torch.zeros(1, M, N, 2, dtype=torch.float16, device="cuda")
    tn.gemm(tn.F16, a, b, c, M, N, K, scale_exp=0, kernel=3)
    ar = torch.view_as_complex(a.double())
    br = torch.view_as_complex(b.double())
    want = torch.matmul(ar[0], br[0])
    got = torch.view_as_complex(c.double())[0]
    rel = (torch.linalg.norm(got - want) / torch.linalg.norm(want)).item()
    assert rel < 3e-4, rel


@pytest.mark.parametrize("M,N,K,batch", [(128, 8, 64, 1), (256, 16, 128, 2), (1024, 128, 512, 1),
                                         (512, 256, 1024, 1), (384, 4, 256, 1), (128, 32, 1 << 17, 1)])
def test_gemm_fp8_tensor_cores(M, N, K, batch):
    # E4M3 operands (kind::f8f6f4), FP32 accumulation, FP16 result; the
    # reference is the FP64 product of the same E4M3 values
    M = 1 << int(np.ceil(np.log2(M)))
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    a = (torch.randn(batch, M, K, 2, generator=g, device="cuda") * 16).to(torch.float8_e4m3fn)
    b = (torch.randn(batch, K, N, 2, generator=g, device="cuda") * 16).to(torch.float8_e4m3fn)
    c = torch.zeros(batch, M, N, 2, dtype=torch.float16, device="cuda")
    mx = torch.zeros(1, dtype=torch.float32, device="cuda")
    e = -int(np.ceil(np.log2(256 * np.sqrt(K)))) - 1
    tn.gemm(tn.FP8, a, b, c, M, N, K, batch=batch, batch_a=True, batch_b=True, scale_exp=e,
            kernel=3, out_max=mx)
    ar = torch.view_as_complex(a.double())
    br = torch.view_as_complex(b.double())
    want = torch.matmul(ar, br) * 2.0 ** e
    got = torch.view_as_complex(c.double())
    mag = torch.matmul(ar.abs(), br.abs()) * 2.0 ** e
    err = (got - want).abs()
    tol = 2 * 2.0 ** -11 * want.abs() + 1e-6 * mag + 2.0 ** -24
    assert bool((err <= tol).all()), float((err / (want.abs() + 1e-9)).max())
    gmax = max(got.real.abs().max().item(), got.imag.abs().max().item())
    assert abs(mx.item() - gmax) <= 1e-6 * gmax


def test_gemm_fp8_rejects_short_k():
    a = torch.zeros(128, 32, 2, dtype=torch.uint8, device="cuda")
    b = torch.zeros(32, 8, 2, dtype=torch.uint8, device="cuda")
    c = torch.zeros(128, 8, 2, dtype=torch.float16, device="cuda")
    with pytest.raises(tn.TnError):
        tn.gemm(tn.FP8, a, b, c, 128, 8, 32, kernel=3)
