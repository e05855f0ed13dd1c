"""Embed, crop and product on a window of y starting at a tuple (Section 4's biased slices),
bit for bit against the oracle: every dtype, windows that leave rows misaligned (element
paths) or aligned (vector paths), windows touching y's far corner, x overhanging y in the
product, NOPAD, empty x, the FFT zero-pad / extract round trip, and a multi-tile case."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1608_00099_gb300 import synth

pytestmark = pytest.mark.gpu

TORCH = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


@pytest.fixture(scope="module")
def tr():
    from paper_1608_00099_gb300 import build, triot
    build.build()
    triot.lib()
    assert torch.cuda.is_available()
    return triot


def values(n, dtype, seed):
    v = synth.normal01(seed, n)
    return orc.from_f64(v, dtype) if dtype != "f64" else v


def dev(a, dtype, shape):
    t = torch.from_numpy(np.ascontiguousarray(a).reshape(shape).copy())
    if dtype in ("bf16", "f16"):
        t = t.view(torch.int16).view(TORCH[dtype])
    return t.cuda()


def host(t, dtype):
    t = t.cpu()
    if dtype in ("bf16", "f16"):
        t = t.view(torch.int16)
    return t.numpy().reshape(-1)


CASES = [
    ((3, 4), (9, 11), (2, 5)),
    ((5, 7, 6), (9, 12, 10), (4, 5, 4)),          # window in y's far corner
    ((8, 8, 8), (16, 16, 16), (4, 4, 4)),         # the FFT centre pad
    ((6, 30, 64), (9, 40, 130), (1, 7, 66)),      # aligned rows (vector path) for 16-bit types
    ((1, 7, 1, 5), (3, 9, 2, 8), (2, 1, 1, 3)),   # unit axes
    ((2, 300, 257), (3, 301, 600), (1, 1, 343)),  # several tiles, odd rows
    ((0, 4), (3, 5), (1, 1)),                     # empty x
]


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_embed_crop_at_bit_exact(tr, dtype, case):
    xs, ys, st = CASES[case]
    xh = values(int(np.prod(xs)), dtype, 700 + case)
    yh = values(int(np.prod(ys)), dtype, 720 + case)
    # embed with the pad
    y = dev(yh, dtype, ys)
    tr.triot_embed_at(dev(xh, dtype, xs), y, st)
    assert host(y, dtype).tobytes() == orc.embed_at(xh, xs, ys, st, dtype).tobytes()
    # NOPAD keeps the rest of y
    y = dev(yh, dtype, ys)
    tr.triot_embed_at(dev(xh, dtype, xs), y, st, flags=1)
    assert host(y, dtype).tobytes() == orc.embed_at(xh, xs, ys, st, dtype, y=yh).tobytes()
    # crop at
    x = torch.empty(xs, dtype=TORCH[dtype], device="cuda")
    tr.triot_crop_at(x, dev(yh, dtype, ys), st)
    assert host(x, dtype).tobytes() == orc.crop_at(yh, xs, ys, st, dtype).tobytes()


PROD_CASES = [
    ((4, 6, 3), (5, 8, 4), (2, 3, 2)),            # x overhangs y on every axis
    ((7, 9), (20, 30), (5, 11)),
    ((3, 40, 70), (5, 50, 200), (1, 3, 100)),
    ((5, 5), (5, 5), (5, 0)),                     # start at y's end: nothing fits
]


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("case", range(len(PROD_CASES)))
def test_product_at_bit_exact(tr, dtype, case):
    xs, ys, st = PROD_CASES[case]
    xh = values(int(np.prod(xs)), dtype, 740 + case)
    yh = values(int(np.prod(ys)), dtype, 760 + case)
    y = dev(yh, dtype, ys)
    tr.triot_product_at(dev(xh, dtype, xs), y, st)
    assert host(y, dtype).tobytes() == orc.product_at(xh, xs, yh, ys, st, dtype).tobytes()


def test_fft_pad_round_trip(tr):
    """Zero-pad x into the centre of a twice-as-large y and extract it again."""
    xs, ys, st = (8,) * 6, (16,) * 6, (4,) * 6
    xh = values(8 ** 6, "f64", 780)
    x = dev(xh, "f64", xs)
    y = torch.full(ys, 7.0, dtype=torch.float64, device="cuda")
    tr.triot_embed_at(x, y, st)
    assert float(y.abs().sum()) == pytest.approx(float(np.abs(xh).sum()), rel=1e-12)
    back = torch.empty(xs, dtype=torch.float64, device="cuda")
    tr.triot_crop_at(back, y, st)
    assert torch.equal(back, x)


# ---------------------------------------------------------------- windows on both sides

VIEWS2 = [
    # ext, x container, x start, y container, y start
    ((3, 4, 5), (6, 7, 9), (2, 1, 3), (5, 8, 7), (1, 4, 0)),
    ((5, 9), (7, 10), (1, 1), (9, 13), (3, 2)),                     # odd starts: element paths
    ((4, 16), (4, 32), (0, 8), (8, 48), (2, 16)),                   # aligned rows: vector paths
    ((2, 3, 4, 5), (2, 3, 4, 5), (0, 0, 0, 0), (4, 6, 8, 10), (2, 3, 4, 5)),
    ((1, 5000), (3, 6000), (2, 17), (2, 9000), (1, 3001)),          # a long row, segmented
    ((0, 4), (3, 4), (1, 0), (2, 8), (0, 4)),                       # empty window
    ((7, 1, 33), (9, 2, 40), (1, 1, 5), (8, 3, 35), (0, 2, 2)),     # a unit axis in the window
]


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("case", range(len(VIEWS2)))
def test_copy_and_product_views_against_oracle(tr, dtype, case):
    ext, xs, xo, ys, yo = VIEWS2[case]
    xh = values(int(np.prod(xs)), dtype, 900 + case)
    yh = values(int(np.prod(ys)), dtype, 950 + case)
    band = 24
    nyy = int(np.prod(ys))
    buf = torch.full((nyy + 2 * band,), -9, dtype=TORCH[dtype], device="cuda")
    y = buf[band:band + nyy].view(ys)
    y.copy_(dev(yh, dtype, ys))
    x = dev(xh, dtype, xs)
    tr.triot_copy_views(ext, x, xo, y, yo)
    want = orc.copy_views(ext, xh, xs, xo, yh, ys, yo, dtype)
    assert host(y, dtype).tobytes() == want.tobytes()
    tr.triot_product_views(ext, x, xo, y, yo)
    want = orc.product_views(ext, xh, xs, xo, want, ys, yo, dtype)
    assert host(y, dtype).tobytes() == want.tobytes()
    sentinel = host(torch.full((1,), -9, dtype=TORCH[dtype], device="cuda"), dtype)[0]
    hb = host(buf, dtype)
    assert np.all(hb[:band] == sentinel) and np.all(hb[band + nyy:] == sentinel)


@pytest.mark.parametrize("dtype", ["f64", "bf16"])
def test_product_support_of_two_pmfs(tr, dtype):
    """Two PMFs on one integer grid with different supports: y *= x over the tuples both
    cover, the rest of y untouched -- the oracle's window product on the intersection."""
    xs, xo = (12, 9, 14), (-3, 5, 2)
    ys, yo = (10, 12, 9), (1, 0, 6)
    xh = values(int(np.prod(xs)), dtype, 61)
    yh = values(int(np.prod(ys)), dtype, 62)
    lo = [max(a, b) for a, b in zip(xo, yo)]
    hi = [min(a + n, b + m) for a, n, b, m in zip(xo, xs, yo, ys)]
    ext = [max(0, h - l) for l, h in zip(lo, hi)]
    want = orc.product_views(ext, xh, xs, [l - a for l, a in zip(lo, xo)], yh, ys,
                             [l - b for l, b in zip(lo, yo)], dtype)
    y = dev(yh, dtype, ys)
    tr.triot_product_support(dev(xh, dtype, xs), xo, y, yo)
    assert host(y, dtype).tobytes() == want.tobytes()
    # disjoint supports: nothing changes
    y2 = dev(yh, dtype, ys)
    tr.triot_product_support(dev(xh, dtype, xs), (100, 0, 0), y2, yo)
    assert host(y2, dtype).tobytes() == yh.tobytes()


def test_views_reject_bad_windows(tr):
    x = torch.zeros((4, 5), device="cuda")
    y = torch.zeros((6, 6), device="cuda")
    with pytest.raises(tr.TriotError):
        tr.triot_copy_views((3, 3), x, (2, 0), y, (0, 0))      # x window leaves x
    with pytest.raises(tr.TriotError):
        tr.triot_product_views((3, 3), x, (0, 0), y, (4, 0))   # y window leaves y
    with pytest.raises(tr.TriotError):
        tr.triot_product_views((2, 2), x, (0, 0), x, (1, 1))   # the same container
