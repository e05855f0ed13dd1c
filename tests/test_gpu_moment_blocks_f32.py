"""f32 / bf16 / f16 moment on tensors whose trailing axes form short blocks.

These shapes take the block-column kernels with f32 sums: chunked blocks of B = 1..16
elements and warp blocks of 128..256 (staged, or read with 16-byte loads when a block is a
whole number of 512-byte rows), one to twenty outer axes (carries through several levels,
jumps that change cold axes), tails that end inside a round, signed, subnormal, non-finite
and unaligned input, windows of every phase.  The reference is the oracle's compensated f64
sum of the stored values (Algorithms 10 and 11); the tolerance is the stated
FP32-accumulation bound, 1e-5 of sum |p[t]| t_i per component (the kernels' own bounds are
about 5.6e-6).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1608_00099_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
TORCH = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


@pytest.fixture(scope="module")
def tr():
    from paper_1608_00099_gb300 import build, triot
    build.build()
    triot.lib()
    assert torch.cuda.is_available()
    return triot


def stored(v, dtype):
    """v rounded to the storage type (the oracle's rounding), as stored bits."""
    return orc.from_f64(v, dtype)


def dev(h, dtype, shape):
    t = torch.from_numpy(np.ascontiguousarray(h).reshape(shape).copy())
    if dtype in ("bf16", "f16"):
        t = t.view(torch.int16).view(TORCH[dtype])
    return t.cuda()


def scale(h, shape, dtype):
    return np.abs(orc.moment(np.abs(orc.to_f64(h, dtype)), shape, "f64"))


def check(got, ref, sc):
    err = np.abs(got - ref)
    assert np.all(err <= TOL * sc + 1e-300), (got, ref, err / np.maximum(sc, 1e-300))


BLOCK_SHAPES = [
    (5,), (16,), (2, 2, 2, 2), (3, 7), (1000, 9), (7, 11, 13), (50, 3, 5), (33, 40, 2, 2, 3),
    (9,) * 6, (17, 19, 23, 14), (4,) * 10, (2,) * 20, (101, 103, 6), (5, 7, 9, 11, 2),
    (3,) * 12, (100003, 10), (31, 37, 41, 8), (3, 5, 7, 4), (2, 3, 1, 5, 1, 3), (61, 67, 11),
    (1, 1, 12), (8191, 1, 1), (999, 15), (3001, 13), (77, 7), (40, 2, 7), (1, 1, 1),
    (7, 2, 128), (3, 5, 256), (1001, 33), (70, 4, 64), (6, 4, 7, 3, 5, 3, 3, 3, 6, 3),
    (16, 16), (2, 128), (9, 15),                # one block: no outer axis
]


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("shape", BLOCK_SHAPES)
def test_block_moment_f32_matches_oracle(tr, shape, dtype):
    n = int(np.prod(shape))
    law = synth.normal01 if n % 2 else synth.uniform01
    h = stored(law(800 + n % 983, n), dtype)
    ref = orc.moment(h, shape, dtype)
    got = tr.triot_moment(dev(h, dtype, shape)).cpu().numpy()
    check(got, ref, scale(h, shape, dtype))


def test_block_moment_f32_d24_all_two(tr):
    """The d=24 workload: 2^24 U(0,1) f32 values of shape (2,)*24 (blocks of 16)."""
    shape = (2,) * 24
    n = 1 << 24
    h = stored(synth.uniform01(1003, n), "f32")
    ref = orc.moment(h, shape, "f32")
    got = tr.triot_moment(dev(h, "f32", shape)).cpu().numpy()
    check(got, ref, scale(h, shape, "f32"))


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_block_moment_f32_wide_range_subnormals_zeros(tr, dtype):
    shape = (40, 31, 16)
    n = int(np.prod(shape))
    rng = np.random.default_rng(n)
    v = rng.standard_normal(n) * 10.0 ** rng.integers(-30, 30, size=n)
    v[:50] = rng.standard_normal(50) * 1e-40      # f32 subnormals
    v[50:70] = 0.0
    v[70:80] = -0.0
    h = stored(v, dtype)
    ref = orc.moment(h, shape, dtype)
    got = tr.triot_moment(dev(h, dtype, shape)).cpu().numpy()
    check(got, ref, scale(h, shape, dtype))


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("bad", [np.inf, -np.inf, np.nan])
def test_block_moment_f32_nonfinite(tr, dtype, bad):
    shape = (20, 30, 9)
    n = int(np.prod(shape))
    v = synth.uniform01(73, n)
    v[3 * 270 + 5 * 9 + 4] = bad   # tuple (3, 5, 4): every component of the tuple is nonzero
    h = stored(v, dtype)
    got = tr.triot_moment(dev(h, dtype, shape)).cpu().numpy()
    ref = orc.moment(h, shape, dtype)
    for g_, r_ in zip(got, ref):
        assert (np.isnan(g_) and np.isnan(r_)) or g_ == r_


@pytest.mark.parametrize("dtype", ["f32", "f16"])
@pytest.mark.parametrize("shape", [(37, 29, 3), (9, 4, 4, 4, 4), (5, 8, 32)])
def test_block_moment_f32_unaligned(tr, dtype, shape):
    n = int(np.prod(shape))
    h = stored(synth.uniform01(74, n), dtype)
    buf = torch.zeros(n + 8, dtype=TORCH[dtype], device="cuda")
    p = buf[1:1 + n].view(shape)
    p.copy_(dev(h, dtype, shape))
    got = tr.triot_moment(p).cpu().numpy()
    check(got, orc.moment(h, shape, dtype), scale(h, shape, dtype))


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_block_moment_f32_point_masses_and_determinism(tr, dtype):
    shape = (13, 11, 7, 5, 3)
    n = int(np.prod(shape))
    for k in [0, 1, 14, 2 * 1155 + 17, n - 1]:
        p = torch.zeros(shape, dtype=TORCH[dtype], device="cuda")
        p.view(-1)[k] = 0.75
        got = tr.triot_moment(p).cpu().numpy()
        t = np.unravel_index(k, shape)
        assert list(got) == [0.75 * x for x in t] + [0.75]
    h = stored(synth.normal01(75, n), dtype)
    a = tr.triot_moment(dev(h, dtype, shape)).cpu().numpy()
    b = tr.triot_moment(dev(h, dtype, shape)).cpu().numpy()
    assert a.tobytes() == b.tobytes()


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
def test_block_moment_empty(tr, dtype):
    tdt = {"f64": torch.float64, **TORCH}[dtype]
    z = tr.triot_moment(torch.empty((3, 0, 2), dtype=tdt, device="cuda")).cpu().numpy()
    assert list(z) == [0.0] * 4
