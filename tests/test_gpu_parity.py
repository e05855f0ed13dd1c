"""GPU parity: every kernel against the CPU oracle, element by element, on seeded inputs.

Embed, crop and products are compared bit for bit (every dtype).  Moments are compared
with the tolerance of their accumulation: f64 input within 1e-12 of the exact value
relative to sum_t |p[t]| * t_i (and to sum |p| for the mass), f32/bf16/f16 input within
1e-5 on the same scale.  All calls go through the C ABI (paper_1608_00099_gb300.triot).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1608_00099_gb300 import synth

pytestmark = pytest.mark.gpu

TORCH = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}
TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 1e-5, "f16": 1e-5}


@pytest.fixture(scope="module")
def tr():
    from paper_1608_00099_gb300 import build, triot
    build.build()
    triot.lib()
    assert torch.cuda.is_available()
    return triot


def host_values(n, dtype, seed, law="normal"):
    """Storage-typed numpy values (bf16/f16 as uint16 bits) from the seeded generators."""
    v = synth.normal01(seed, n) if law == "normal" else synth.uniform01(seed, n)
    if dtype == "f64":
        return v
    if dtype == "f32":
        return v.astype(np.float32)
    return orc.from_f64(v, dtype)


def to_dev(a, dtype, shape):
    t = torch.from_numpy(np.ascontiguousarray(a).reshape(shape).copy())
    if dtype in ("bf16", "f16"):
        t = t.view(torch.int16).view(TORCH[dtype])
    return t.cuda()


def to_host(t, dtype):
    t = t.detach().cpu().contiguous()
    if dtype in ("bf16", "f16"):
        return t.view(torch.int16).numpy().view(np.uint16).reshape(-1)
    return t.numpy().reshape(-1)


def misaligned(shape, dtype):
    """A contiguous device tensor whose data starts one element past a 16-byte boundary."""
    n = int(np.prod(shape))
    buf = torch.empty(n + 8, dtype=TORCH[dtype], device="cuda")
    return buf[1:1 + n].view(shape)


def moment_scale(p_host, shape, dtype):
    """sum |p| t_i and sum |p| from the oracle on |p| (the scale of the tolerance)."""
    w = np.abs(orc.to_f64(p_host, dtype))
    return np.abs(orc.moment(w, shape, "f64"))


def check_moment(got, ref, scale, tol):
    err = np.abs(got - ref)
    bound = tol * scale + 1e-300
    assert np.all(err <= bound), (got, ref, err / np.maximum(scale, 1e-300))


# ---------------------------------------------------------------- embed / crop

EMBED_SHAPES = [
    ((8,) * 6, (10,) * 6),                 # the small f64 d=6 workload
    ((3, 5), (4, 7)),
    ((1000,), (1037,)),                    # rank 1, ragged tail
    ((9, 9, 9), (11, 10, 11)),
    ((2,) * 10, (3,) * 6 + (2,) * 4),      # high rank, tiny extents, merged rows
    ((5, 1, 7), (6, 1, 9)),
    ((17, 33, 65), (17, 40, 65)),          # merged inner axes
    ((3, 3000), (4, 9001)),                # row segments longer than a tile
    ((0, 4), (3, 4)),                      # empty x: y is all pad
    ((1,), (1,)),
]


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("shapes", EMBED_SHAPES)
def test_embed_and_crop_bit_exact(tr, dtype, shapes):
    xs, ys = shapes
    nx = int(np.prod(xs))
    xh = host_values(nx, dtype, 11 + nx)
    ref = orc.embed(xh, xs, ys, dtype)
    x = to_dev(xh, dtype, xs)
    y = torch.full(ys, 7, dtype=TORCH[dtype], device="cuda")   # stale values must be overwritten
    tr.triot_embed(x, y)
    assert to_host(y, dtype).tobytes() == ref.tobytes()
    x2 = torch.full(xs, 3, dtype=TORCH[dtype], device="cuda")
    tr.triot_crop(x2, y)
    assert to_host(x2, dtype).tobytes() == xh.tobytes()


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_embed_crop_misaligned_and_nopad(tr, dtype):
    xs, ys = (7, 13, 6), (9, 16, 8)
    xh = host_values(int(np.prod(xs)), dtype, 5)
    ref = orc.embed(xh, xs, ys, dtype)
    x = misaligned(xs, dtype)
    x.copy_(to_dev(xh, dtype, xs))
    y = misaligned(ys, dtype)
    y.fill_(5)
    tr.triot_embed(x, y)
    assert to_host(y, dtype).tobytes() == ref.tobytes()
    x2 = misaligned(xs, dtype)
    tr.triot_crop(x2, y)
    assert to_host(x2, dtype).tobytes() == xh.tobytes()
    # NOPAD: only x's tuples are written
    y3 = torch.zeros(ys, dtype=TORCH[dtype], device="cuda")
    y3.view(-1)[-1] = 9   # a pad element that must survive
    tr.triot_embed(x, y3, flags=tr.EMBED_NOPAD)
    h = to_host(y3, dtype).copy()
    expect = ref.copy()
    expect[-1] = to_host(torch.full((1,), 9, dtype=TORCH[dtype]).cuda(), dtype)[0]
    assert h.tobytes() == expect.tobytes()


def test_embed_guard_band_untouched(tr):
    xs, ys = (9, 9, 9, 9), (11, 10, 11, 10)
    n = int(np.prod(ys))
    buf = torch.full((n + 64,), -1.0, dtype=torch.float64, device="cuda")
    y = buf[32:32 + n].view(ys)
    x = to_dev(host_values(int(np.prod(xs)), "f64", 3), "f64", xs)
    tr.triot_embed(x, y)
    h = buf.cpu().numpy()
    assert np.all(h[:32] == -1.0) and np.all(h[32 + n:] == -1.0)


def _guarded(shape, dtype, fill, band=40):
    """A tensor of `shape` inside a buffer with `band` sentinel elements on each side."""
    n = int(np.prod(shape))
    buf = torch.full((n + 2 * band,), fill, dtype=TORCH[dtype], device="cuda")
    return buf, buf[band:band + n].view(shape)


def _band_intact(buf, n, dtype, fill, band=40):
    h = to_host(buf, dtype)
    f = to_host(torch.full((1,), fill, dtype=TORCH[dtype]).cuda(), dtype)[0]
    return np.all(h[:band] == f) and np.all(h[band + n:] == f)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("shapes", [((9,) * 4, (12, 8, 12, 8)), ((7, 13, 6), (9, 16, 8)), ((3, 3000), (4, 9001))])
def test_product_and_crop_guard_bands_untouched(tr, dtype, shapes):
    xs, ys = shapes
    xh = host_values(int(np.prod(xs)), dtype, 41, law="uniform")
    yh = host_values(int(np.prod(ys)), dtype, 42)
    x = to_dev(xh, dtype, xs)
    ybuf, y = _guarded(ys, dtype, -3)
    y.copy_(to_dev(yh, dtype, ys))
    tr.triot_product(x, y)
    assert to_host(y, dtype).tobytes() == orc.product(xh, xs, yh, ys, dtype).tobytes()
    assert _band_intact(ybuf, int(np.prod(ys)), dtype, -3)
    cs = tuple(min(a, b) for a, b in zip(xs, ys))
    cbuf, c = _guarded(cs, dtype, -5)
    tr.triot_crop(c, y)
    ref = orc.crop(orc.product(xh, xs, yh, ys, dtype), cs, ys, dtype)
    assert to_host(c, dtype).tobytes() == ref.tobytes()
    assert _band_intact(cbuf, int(np.prod(cs)), dtype, -5)


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16"])
def test_views_guard_bands_untouched(tr, dtype):
    xs, ys, st = (5, 6, 7), (9, 11, 13), (2, 3, 5)
    xh = host_values(int(np.prod(xs)), dtype, 43, law="uniform")
    ny = int(np.prod(ys))
    x = to_dev(xh, dtype, xs)
    ybuf, y = _guarded(ys, dtype, -7)
    tr.triot_embed_at(x, y, st)
    assert to_host(y, dtype).tobytes() == orc.embed_at(xh, xs, ys, st, dtype).tobytes()
    assert _band_intact(ybuf, ny, dtype, -7)
    xbuf, x2 = _guarded(xs, dtype, -9)
    tr.triot_crop_at(x2, y, st)
    assert to_host(x2, dtype).tobytes() == xh.tobytes()
    assert _band_intact(xbuf, int(np.prod(xs)), dtype, -9)
    yh = to_host(y, dtype).copy()
    tr.triot_product_at(x, y, st)
    assert to_host(y, dtype).tobytes() == orc.product_at(xh, xs, yh, ys, st, dtype).tobytes()
    assert _band_intact(ybuf, ny, dtype, -7)


# ---------------------------------------------------------------- product

PROD_SHAPES = [
    ((9,) * 4, (12, 8, 12, 8)),
    ((5, 7), (3, 9)),
    ((4000,), (3001,)),
    ((2,) * 12, (3,) * 8 + (2,) * 4),
    ((6, 1, 5), (4, 3, 7)),                # intersection axis of extent 1 with strided x
    ((3, 2), (3, 1)),                      # unit inner axis in the intersection
    ((31, 17, 9), (33, 17, 9)),
    ((2, 5000), (2, 7000)),
]


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("shapes", PROD_SHAPES)
def test_product_bit_exact(tr, dtype, shapes):
    xs, ys = shapes
    xh = host_values(int(np.prod(xs)), dtype, 21, law="uniform")
    yh = host_values(int(np.prod(ys)), dtype, 22)
    ref = orc.product(xh, xs, yh, ys, dtype)
    x = to_dev(xh, dtype, xs)
    y = to_dev(yh, dtype, ys)
    tr.triot_product(x, y)
    assert to_host(y, dtype).tobytes() == ref.tobytes()


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16"])
def test_product_misaligned(tr, dtype):
    xs, ys = (10, 6, 9), (8, 8, 12)
    xh = host_values(int(np.prod(xs)), dtype, 23)
    yh = host_values(int(np.prod(ys)), dtype, 24)
    ref = orc.product(xh, xs, yh, ys, dtype)
    x = misaligned(xs, dtype)
    x.copy_(to_dev(xh, dtype, xs))
    y = misaligned(ys, dtype)
    y.copy_(to_dev(yh, dtype, ys))
    tr.triot_product(x, y)
    assert to_host(y, dtype).tobytes() == ref.tobytes()


def test_product_bf16_tiny_and_special_values(tr):
    rng = np.random.default_rng(9)
    mags = 2.0 ** rng.integers(-140, 127, size=4096) * (1 + rng.random(4096))
    sgn = np.where(rng.random(4096) < 0.5, -1.0, 1.0)
    a = orc.from_f64(mags * sgn, "bf16")
    b = orc.from_f64(2.0 ** rng.integers(-140, 0, size=4096) * (1 + rng.random(4096)), "bf16")
    a[:6] = orc.from_f64(np.array([0.0, -0.0, np.inf, 3.0, 2.0 ** -133, 1e38]), "bf16")
    b[:6] = orc.from_f64(np.array([5.0, 2.0, 2.0, 0.0, 0.5, 1e10]), "bf16")
    ref = orc.product(a, (4096,), b, (4096,), "bf16")
    x = to_dev(a, "bf16", (4096,))
    y = to_dev(b, "bf16", (4096,))
    tr.triot_product(x, y)
    got = to_host(y, "bf16")
    assert got.tobytes() == ref.tobytes()


def test_product_f16_subnormals(tr):
    rng = np.random.default_rng(10)
    a = (rng.random(5000) * 1e-3).astype(np.float16).view(np.uint16)
    b = (rng.random(5000) * 1e-2).astype(np.float16).view(np.uint16)
    ref = orc.product(a, (5000,), b, (5000,), "f16")
    y = to_dev(b, "f16", (5000,))
    tr.triot_product(to_dev(a, "f16", (5000,)), y)
    assert to_host(y, "f16").tobytes() == ref.tobytes()


# ---------------------------------------------------------------- moment

MOMENT_SHAPES = [(9,) * 5, (7, 3), (100000,), (2,) * 16, (3, 1, 4, 1, 5), (6, 4, 7, 3, 5, 6, 7, 3, 7, 3),
                 (1,), (1, 1, 3), (13, 17, 19), (5000, 3), (3, 5000)]


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("shape", MOMENT_SHAPES)
def test_moment_within_tolerance(tr, dtype, shape):
    n = int(np.prod(shape))
    ph = host_values(n, dtype, 31 + n)
    ref = orc.moment(ph, shape, dtype)
    got = tr.triot_moment(to_dev(ph, dtype, shape)).cpu().numpy()
    check_moment(got, ref, moment_scale(ph, shape, dtype), TOL[dtype])


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_moment_point_mass_and_determinism(tr, dtype):
    shape = (9, 9, 9, 9)
    n = int(np.prod(shape))
    for k in [0, 4321, n - 1]:
        p = torch.zeros(shape, dtype=TORCH[dtype], device="cuda")
        p.view(-1)[k] = 1.0
        m = tr.triot_moment(p).cpu().numpy()
        assert list(m) == [float(v) for v in np.unravel_index(k, shape)] + [1.0]
    ph = host_values(n, dtype, 77)
    p = to_dev(ph, dtype, shape)
    a = tr.triot_moment(p).cpu().numpy()
    b = tr.triot_moment(p).cpu().numpy()
    assert a.tobytes() == b.tobytes()


def test_moment_f64_wide_dynamic_range_and_subnormals(tr):
    shape = (40, 31, 17)
    n = int(np.prod(shape))
    rng = np.random.default_rng(12)
    v = rng.standard_normal(n) * 10.0 ** rng.integers(-300, 300, size=n)
    v[:50] = rng.standard_normal(50) * 1e-310       # subnormals
    v[50:60] = 0.0
    ref = orc.moment(v, shape, "f64")
    got = tr.triot_moment(torch.from_numpy(v.reshape(shape)).cuda()).cpu().numpy()
    check_moment(got, ref, moment_scale(v, shape, "f64"), 1e-12)


def _same_moment_with_specials(got, ref, scale, tol):
    """Non-finite components must match the oracle's class exactly (the same infinity, or
    NaN on both sides); finite ones within the tolerance."""
    for g, r, sc in zip(got, ref, scale):
        if np.isnan(r):
            assert np.isnan(g), (got, ref)
        elif np.isinf(r):
            assert g == r, (got, ref)
        else:
            assert np.isfinite(g) and abs(g - r) <= tol * sc + 1e-300, (got, ref)


@pytest.mark.parametrize("case", ["inf", "inf_zero_digit", "both_infinities", "nan", "neg_inf_signed"])
@pytest.mark.parametrize("shape", [(20, 33), (9, 9, 9, 9), (40, 7, 3)])
def test_moment_f64_nonfinite_against_oracle(tr, case, shape):
    n = int(np.prod(shape))
    v = synth.uniform01(5, n)
    if case == "inf":
        v[n // 2 + 1] = np.inf
    elif case == "inf_zero_digit":
        v[0] = np.inf                      # tuple (0, ..., 0): inf * 0 is NaN in every moment
    elif case == "both_infinities":
        v[n // 3] = np.inf
        v[2 * n // 3] = -np.inf
    elif case == "nan":
        v[n - 1] = np.nan
    else:
        v = v - 0.5
        v[n // 5] = -np.inf
    ref = orc.moment(v, shape, "f64")
    got = tr.triot_moment(torch.from_numpy(v.reshape(shape)).cuda()).cpu().numpy()
    scale = moment_scale(np.where(np.isfinite(v), v, 0.0), shape, "f64")
    assert not np.all(np.isfinite(ref))
    _same_moment_with_specials(got, ref, scale, 1e-12)


def test_moment_unaligned_input(tr):
    for dtype in ("f64", "f32", "bf16"):
        shape = (37, 29)
        ph = host_values(37 * 29, dtype, 8)
        p = misaligned(shape, dtype)
        p.copy_(to_dev(ph, dtype, shape))
        got = tr.triot_moment(p).cpu().numpy()
        check_moment(got, orc.moment(ph, shape, dtype), moment_scale(ph, shape, dtype), TOL[dtype])


def test_moment_empty_and_workspace_errors(tr):
    m = tr.triot_moment(torch.empty((3, 0, 2), dtype=torch.float32, device="cuda")).cpu().numpy()
    assert np.all(m == 0.0) and m.size == 4
    p = torch.ones((64, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(tr.TriotError):
        tr.triot_moment(p, workspace=torch.empty(1, dtype=torch.float64, device="cuda"))


# ---------------------------------------------------------------- batched pipeline

def _batch(tr, pairs, mode, plain=False, dtype="f32"):
    xs_h = synth.batch_x_values(pairs)
    xs, ys, outs = [], [], []
    for pr, xh in zip(pairs, xs_h):
        xv = xh.astype(np.float32) if dtype == "f32" else orc.from_f64(xh, dtype) if dtype != "f64" else xh
        xs.append(to_dev(xv, dtype, pr.xshape))
        ys.append(torch.full(pr.yshape, 3, dtype=TORCH[dtype], device="cuda"))
        outs.append(torch.zeros(len(pr.xshape) + 1, dtype=torch.float64, device="cuda"))
    plan = tr.BatchPlan(xs, ys, outs, mode=mode)
    if plain:
        plan.run_plain()
    else:
        plan.run()
        plan.run()   # graph replay: same result
    torch.cuda.synchronize()
    return plan, xs, ys, outs


@pytest.mark.parametrize("mode", ["fused", "phased", "plain"])
@pytest.mark.parametrize("dtype", ["f32", "bf16", "f64"])
def test_batch_small_against_oracle(tr, mode, dtype):
    pairs = synth.config_batch_shapes(npairs=48, cap_log2=16)
    m = {"fused": tr.BATCH_FUSED, "phased": tr.BATCH_PHASED, "plain": tr.BATCH_FUSED}[mode]
    plan, xs, ys, outs = _batch(tr, pairs, m, plain=(mode == "plain"), dtype=dtype)
    for pr, x, y, o in zip(pairs, xs, ys, outs):
        xh = to_host(x, dtype)
        ye = orc.embed(xh, pr.xshape, pr.yshape, dtype)
        ye = orc.product(xh, pr.xshape, ye, pr.yshape, dtype)
        assert to_host(y, dtype).tobytes() == ye.tobytes()
        ref = orc.moment(ye, pr.yshape, dtype)
        check_moment(o.cpu().numpy(), ref, moment_scale(ye, pr.yshape, dtype), 1e-5 if dtype != "f64" else 1e-12)
    plan.close()
    assert tr.triot_device_status() == 0
