"""The Sec. 3.2 codec kernels (tn_encode / tn_decode) against the oracle
(oracle/codec.py): codes bit-exact where the codes come from exactly rounded
FP32 operations (half, int4), and within one step where the int8 kind's
x^0.2 (powf) may differ by an ulp from the host's; scales, zeros and
decoded values against the oracle's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
from oracle import codec  # noqa: E402
import paper_2407_00769_gb300 as tn  # noqa: E402

pytestmark = pytest.mark.gpu
KIND = {"half": tn.CODEC_HALF, "int8": tn.CODEC_INT8, "int4": tn.CODEC_INT4}


def _data(n, seed, dist="normal"):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n) if dist == "normal" else rng.uniform(-5, 7, size=n)
    return x.astype(np.float32)


@pytest.mark.parametrize("kind,group,n", [("int4", 128, 1 << 16), ("int4", 1024, 1 << 14), ("int4", 128, 128),
                                          ("half", 0, 1 << 16), ("half", 0, 1000), ("int8", 0, 1 << 16),
                                          ("int8", 0, 7)])
def test_codec_against_oracle(kind, group, n):
    x = _data(n, n + group, "uniform" if kind == "int8" else "normal")
    xd = torch.from_numpy(x).cuda()
    codes, scale, zero = tn.encode(KIND[kind], xd, group)
    want, ws, wz = codec.encode(x, kind, group)
    s, z = scale.cpu().numpy(), zero.cpu().numpy()
    if kind == "int4":
        got = codec.unpack_int4(codes.cpu().numpy())
        assert np.array_equal(s, ws) and np.array_equal(z, wz)
        assert np.array_equal(got, want)
    elif kind == "half":
        got = codes.cpu().numpy()
        assert np.array_equal(s, ws) and np.array_equal(z, wz)
        assert np.array_equal(got.view(np.uint16), want.view(np.uint16))
    else:
        got = codes.cpu().numpy().astype(np.int32)
        assert np.allclose(s, ws, rtol=1e-6) and np.allclose(z, wz, rtol=1e-6, atol=1e-6)
        diff = np.abs(got - want)
        assert diff.max() <= 1 and np.mean(diff > 0) <= 1e-3
    back = tn.decode(KIND[kind], codes, scale, zero, n, group).cpu().numpy().astype(np.float64)
    ref = codec.decode(got, s, z, kind, group)
    assert np.allclose(back, ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())


def test_codec_constant_group_and_rejections():
    x = torch.full((256,), 3.0, dtype=torch.float32, device="cuda")
    codes, scale, zero = tn.encode(tn.CODEC_INT4, x, 128)
    assert torch.allclose(tn.decode(tn.CODEC_INT4, codes, scale, zero, 256, 128), x)
    with pytest.raises(tn.TnError):
        tn.encode(tn.CODEC_INT4, x[:200], 100)
    with pytest.raises(tn.TnError):
        tn.encode(tn.CODEC_INT8, x, 128)
