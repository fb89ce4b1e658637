"""Pins of the codec oracle (oracle/codec.py, Sec. 3.2 Eq. 1, Table 1)."""
import numpy as np
import pytest

from oracle import codec


def test_integer_group_is_reproduced_exactly():
    x = np.arange(16, dtype=np.float32)               # the int4 range itself
    codes, scale, zero = codec.encode(x, "int4", group=16)
    assert codes.tolist() == list(range(16))
    assert scale.tolist() == [1.0] and zero.tolist() == [0.0]
    assert np.array_equal(codec.decode(codes, scale, zero, "int4", group=16), x)


@pytest.mark.parametrize("kind,group", [("int4", 128), ("int8", 0), ("half", 0), ("int4", 32)])
def test_group_extremes_map_to_the_range_ends(kind, group):
    rng = np.random.default_rng(1)
    x = rng.standard_normal(1024).astype(np.float32) * 3
    codes, scale, zero = codec.encode(x, kind, group)
    q_min, q_max, _, _ = codec.KINDS[kind]
    g = x.size if group == 0 else group
    c = np.asarray(codes, dtype=np.float64).reshape(-1, g)
    xs = x.reshape(-1, g)
    for i in range(c.shape[0]):
        assert c[i, np.argmin(xs[i])] == pytest.approx(q_min, abs=1e-3 * abs(q_min) + 1e-6)
        assert c[i, np.argmax(xs[i])] == pytest.approx(q_max, abs=1e-3 * abs(q_max) + 1e-6)


@pytest.mark.parametrize("kind,group", [("int4", 128), ("int8", 0)])
def test_round_trip_within_half_a_step(kind, group):
    # in the transformed domain the rounding moves a value by at most half
    # a quantization step, 0.5 / scale
    rng = np.random.default_rng(2)
    x = rng.standard_normal(4096).astype(np.float32)
    codes, scale, zero = codec.encode(x, kind, group)
    _, _, exp, _ = codec.KINDS[kind]
    back = codec.decode(codes, scale, zero, kind, group)
    g = x.size if group == 0 else group
    yt = codec.transform(x, exp).astype(np.float64).reshape(-1, g)
    yb = (np.sign(back) * np.abs(back) ** exp).reshape(-1, g)
    step = 0.5 / scale.astype(np.float64)[:, None]
    assert np.all(np.abs(yt - yb) <= step * (1 + 1e-5) + 1e-7)
    if exp == 1.0:
        assert np.all(np.abs(x.astype(np.float64).reshape(-1, g) - back.reshape(-1, g)) <= step * (1 + 1e-5) + 1e-7)


def test_exp_is_odd_and_constant_groups_survive():
    x = np.array([-8.0, -1.0, 0.0, 1.0, 8.0], dtype=np.float32)
    y = codec.transform(x, 0.2)
    assert y[0] == -y[4] and y[1] == -1.0 and y[2] == 0.0 and y[3] == 1.0
    assert y[4] == pytest.approx(8.0 ** 0.2, rel=1e-6)
    c = np.full(64, 2.5, dtype=np.float32)
    codes, scale, zero = codec.encode(c, "int4", group=64)
    assert np.allclose(codec.decode(codes, scale, zero, "int4", group=64), 2.5)


def test_int4_packing_round_trip():
    rng = np.random.default_rng(3)
    codes = rng.integers(0, 16, size=256)
    packed = codec.pack_int4(codes)
    assert packed.size == 128 and packed[0] == (codes[0] | (codes[1] << 4))
    assert np.array_equal(codec.unpack_int4(packed), codes)
