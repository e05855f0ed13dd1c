"""Pins of the CPU oracle against what the paper and mathematics fix.

Each check compares the oracle with something other than itself: the value the
paper prints for its worked example, closed forms, numpy/torch library routines
and brute force on tiny inputs.  No GPU is used.
"""
import itertools
import os

import numpy as np
import pytest
import torch

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

SMALL_SHAPES = [(1,), (5,), (3, 4), (2, 3, 4), (4, 1, 3), (2, 2, 2, 2), (3, 1, 1, 2), (1, 4, 2, 3)]


def _read_golden(name):
    rec = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            rec[key] = vals
    return rec


# ---------------------------------------------------------------- Section 1 / Alg 2

def test_worked_example_flat_index(orc):
    g = _read_golden("flat_index_worked_example.txt")
    shape = [int(v) for v in g["shape"]]
    tup = [int(v) for v in g["tuple"]]
    printed = sum(int(np.prod([int(f) for f in term.split("*")])) for term in g["terms"])
    assert printed == int(g["flat"][0]) == 651
    assert orc.tuple_to_index(tup, shape) == 651
    # column-major would give 398; the oracle is row-major
    assert int(np.ravel_multi_index(tup, shape, order="F")) == 398


@pytest.mark.parametrize("shape", SMALL_SHAPES + [(4, 9, 7, 5)])
def test_horner_equals_explicit_sum_and_numpy(orc, shape):
    d = len(shape)
    for tup in itertools.product(*[range(s) for s in shape]):
        explicit = sum(tup[i] * int(np.prod(shape[i + 1:])) for i in range(d))
        assert orc.tuple_to_index(tup, shape) == explicit
        assert explicit == int(np.ravel_multi_index(tup, shape))


def test_horner_random_large(orc):
    rng = np.random.default_rng(7)
    for _ in range(200):
        d = int(rng.integers(1, 25))
        shape = [int(v) for v in rng.integers(1, 6, size=d)]
        tup = [int(rng.integers(0, s)) for s in shape]
        assert orc.tuple_to_index(tup, shape) == int(np.ravel_multi_index(tup, shape))


# ---------------------------------------------------------------- Alg 3

@pytest.mark.parametrize("shape", SMALL_SHAPES)
def test_advance_tuple_lexicographic(orc, shape):
    t = [0] * len(shape)
    for expect in itertools.product(*[range(s) for s in shape]):
        assert tuple(t) == expect
        t = orc.advance_tuple(t, shape)
    # one step past the last tuple carries into axis 0 only
    assert t[0] == shape[0] and all(v == 0 for v in t[1:])


@pytest.mark.parametrize("shape", [(3, 4, 5), (2,) * 10, (7, 3, 2, 5), (9,) * 5])
def test_enumerate_kth_tuple_is_k_and_carry_mean(orc, shape):
    n = int(np.prod(shape))
    idx, changed = orc.enumerate_indices(shape)
    assert np.array_equal(idx, np.arange(n, dtype=np.uint64))
    # axis i changes n / prod_{j>i} s_j times over a full pass (Section 1's argument that
    # the mean carry count is a geometric-series constant)
    expect = sum(1.0 / float(np.prod(shape[i + 1:])) for i in range(len(shape)))
    assert float(changed.mean()) == pytest.approx(expect, rel=1e-12)
    assert float(changed.mean()) < 1.0 / (1.0 - 1.0 / min(shape)) + 1e-12


# ---------------------------------------------------------------- Alg 4 / Alg 12

@pytest.mark.parametrize("pair", [((3, 4), (5, 6)), ((2, 3, 4), (2, 5, 4)), ((4, 9, 7, 5), (5, 9, 8, 6)),
                                  ((1, 3, 1), (2, 4, 3))])
def test_reindex_equals_unravel_ravel(orc, pair):
    s, s2 = pair
    for k in range(int(np.prod(s))):
        t = np.unravel_index(k, s)
        assert orc.reindex(k, s, s2) == int(np.ravel_multi_index(t, s2))


def test_reindex_pow2_equals_reindex_on_benchmark1_shapes(orc):
    # benchmark 1 shapes (Section 3): (2^10, 2^9, 2^8) and (2^9, 2^9, 2^5)
    small, big = (2 ** 9, 2 ** 9, 2 ** 5), (2 ** 10, 2 ** 9, 2 ** 8)
    ls, lb = [9, 9, 5], [10, 9, 8]
    rng = np.random.default_rng(3)
    for k in list(rng.integers(0, int(np.prod(small)), size=2000)) + [0, int(np.prod(small)) - 1]:
        k = int(k)
        r = orc.reindex(k, small, big)
        assert r == orc.reindex_pow2(k, ls, lb)
        assert r == int(np.ravel_multi_index(np.unravel_index(k, small), big))


# ---------------------------------------------------------------- number formats

def _all_bf16_finite():
    """All non-negative finite bf16 values (bit patterns 0x0000..0x7F7F) as float64."""
    bits = np.arange(0, 0x7F80, dtype=np.uint32)
    vals = (bits << 16).view(np.float32).astype(np.float64)
    return bits.astype(np.uint16), vals


def _bf16_brute(v, bits, vals):
    """Nearest bf16 to v by exhaustive search, ties to the even bit pattern; overflow
    to infinity at and beyond max + half an ulp = (2 - 2^-8) * 2^127."""
    sign = 0x8000 if np.signbit(v) else 0
    mag = abs(float(v))
    if mag >= (2.0 - 2.0 ** -8) * 2.0 ** 127:
        return sign | 0x7F80
    dist = np.abs(vals - mag)
    cand = bits[dist == dist.min()]
    if len(cand) > 1:
        cand = [c for c in cand if (int(c) & 1) == 0]
    return sign | int(cand[0])


def test_round_to_bf16_brute_force(orc):
    bits, vals = _all_bf16_finite()
    rng = np.random.default_rng(11)
    samples = list(rng.standard_normal(300) * 10.0 ** rng.integers(-40, 39, size=300))
    # exact ties between consecutive bf16 values, normal and subnormal
    for b in [0x3F80, 0x3F81, 0x0001, 0x0002, 0x007F, 0x0080, 0x7F7E, 0x4049]:
        lo = float((np.uint32(b) << 16).view(np.float32))
        hi = float((np.uint32(b + 1) << 16).view(np.float32))
        samples += [(lo + hi) / 2.0, -(lo + hi) / 2.0, lo + (hi - lo) * 0.4999, lo + (hi - lo) * 0.5001]
    samples += [0.0, -0.0, 2.0 ** -134, 2.0 ** -134 * 1.0000001, 2.0 ** -135, 3.3e38, 3.4e38, -1e39]
    for v in samples:
        got = orc.round_to(v, "bf16")
        assert got == _bf16_brute(float(v), bits, vals), (v, hex(got))


def test_round_to_f16_equals_numpy(orc):
    rng = np.random.default_rng(12)
    vals = np.concatenate([rng.standard_normal(3000) * 10.0 ** rng.integers(-9, 6, size=3000),
                           np.array([65504.0, 65519.99, 65520.0, 70000.0, 2.0 ** -24, 2.0 ** -25,
                                     2.0 ** -25 * 1.0000001, 3 * 2.0 ** -26, 2.0 ** -14, 0.0, -0.0,
                                     np.inf, -np.inf])])
    # exact ties between consecutive halves
    h = np.arange(0, 0x7BFF, 37, dtype=np.uint16)
    lo = h.view(np.float16).astype(np.float64)
    hi = (h + 1).view(np.float16).astype(np.float64)
    vals = np.concatenate([vals, (lo + hi) / 2.0])
    with np.errstate(over="ignore"):
        expect = vals.astype(np.float16).view(np.uint16)
    got = np.array([orc.round_to(float(v), "f16") for v in vals], dtype=np.uint16)
    assert np.array_equal(got, expect)
    assert np.array_equal(orc.from_f64(vals, "f16"), expect)


def test_round_to_f32_equals_numpy(orc):
    rng = np.random.default_rng(13)
    vals = rng.standard_normal(3000) * 10.0 ** rng.integers(-45, 38, size=3000)
    vals = np.concatenate([vals, [3.4028235677973366e38, 3.5e38, 1e-45, 7e-46, 0.0, -0.0]])
    with np.errstate(over="ignore"):
        expect = vals.astype(np.float32)
    got = orc.from_f64(vals, "f32")
    assert np.array_equal(got.view(np.uint32), expect.view(np.uint32))


def test_widening_matches_libraries(orc):
    h = np.arange(0, 1 << 16, dtype=np.uint16)
    f16 = h.view(np.float16).astype(np.float64)
    got = orc.to_f64(h, "f16")
    fin = np.isfinite(f16)
    assert np.array_equal(got[fin], f16[fin]) and np.all(np.isnan(got[~fin]) == np.isnan(f16[~fin]))
    bf = torch.from_numpy(h.view(np.int16).copy()).view(torch.bfloat16).to(torch.float64).numpy()
    got = orc.to_f64(h, "bf16")
    fin = np.isfinite(bf)
    assert np.array_equal(got[fin], bf[fin])


# ---------------------------------------------------------------- embed / crop

EMBED_CASES = [((3,), (7,)), ((2, 3), (4, 5)), ((2, 3, 4), (2, 5, 4)), ((1, 4, 2), (3, 4, 5)),
               ((3, 3, 3, 3), (4, 5, 3, 6)), ((0, 2), (3, 4)), ((2, 2), (2, 2))]


def _np_embed(x, xs, ys, dt):
    y = np.zeros(ys, dtype=x.dtype)
    y[tuple(slice(0, s) for s in xs)] = x.reshape(xs)
    return y.reshape(-1)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("case", EMBED_CASES)
def test_embed_crop_against_numpy_slicing(orc, dtype, case):
    xs, ys = case
    n = int(np.prod(xs))
    rng = np.random.default_rng(n + len(ys))
    if dtype in ("bf16", "f16"):
        x = rng.integers(1, 0x7BFF, size=n).astype(np.uint16)
    else:
        x = rng.standard_normal(n).astype(np.float64 if dtype == "f64" else np.float32)
    y = orc.embed(x, xs, ys, dtype)
    ref = _np_embed(x, xs, ys, dtype)
    assert y.tobytes() == ref.tobytes()
    # crop of the embedded tensor is the identity, bit for bit
    assert orc.crop(y, xs, ys, dtype).tobytes() == x.tobytes()
    # pad region is exactly +0 bits
    mask = np.ones(ys, dtype=bool)
    mask[tuple(slice(0, s) for s in xs)] = False
    assert not y.view(np.uint8).reshape(int(np.prod(ys)), -1)[mask.reshape(-1)].any()


def test_embed_threads_and_window(orc):
    xs, ys = (9, 5, 4), (11, 6, 7)
    x = np.arange(1, 1 + int(np.prod(xs)), dtype=np.float64)
    y1 = orc.embed(x, xs, ys, "f64", nthreads=1)
    y4 = orc.embed(x, xs, ys, "f64", nthreads=4)
    assert y1.tobytes() == y4.tobytes()
    for b, c in [(0, 10), (13, 100), (0, y1.size), (y1.size - 7, 7)]:
        assert orc.embed_window(x, xs, ys, b, c, "f64").tobytes() == y1[b:b + c].tobytes()


# ---------------------------------------------------------------- product

PROD_CASES = [((5,), (3,)), ((3, 4), (5, 2)), ((2, 3, 4), (3, 2, 5)), ((4, 4), (4, 4)),
              ((9, 9, 9), (12, 8, 12)), ((1, 3, 2), (2, 3, 1)), ((0, 3), (2, 3))]


def _np_product(x, xs, y, ys, dt):
    I = tuple(min(a, b) for a, b in zip(xs, ys))
    yy = y.reshape(ys).copy()
    sl = tuple(slice(0, s) for s in I)
    yy[sl] = yy[sl] * x.reshape(xs)[sl]
    return yy.reshape(-1)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("case", PROD_CASES)
def test_product_float_against_numpy(orc, dtype, case):
    xs, ys = case
    rng = np.random.default_rng(int(np.prod(xs)) + 3)
    nd = np.float64 if dtype == "f64" else np.float32
    x = rng.standard_normal(int(np.prod(xs))).astype(nd)
    y = rng.standard_normal(int(np.prod(ys))).astype(nd)
    got = orc.product(x, xs, y, ys, dtype)
    assert got.tobytes() == _np_product(x, xs, y, ys, dtype).tobytes()


def test_product_f16_against_numpy_half(orc):
    xs, ys = (6, 7, 5), (5, 9, 5)
    rng = np.random.default_rng(5)
    x = (rng.standard_normal(int(np.prod(xs))) * 30).astype(np.float16)
    y = (rng.standard_normal(int(np.prod(ys))) * 30).astype(np.float16)
    # include subnormal and overflowing products
    x[:4] = np.array([1e-4, 3e-5, 300.0, 6e-8], dtype=np.float16)
    y[:4] = np.array([1e-4, 2e-3, 300.0, 0.5], dtype=np.float16)
    got = orc.product(x.view(np.uint16), xs, y.view(np.uint16), ys, "f16")
    with np.errstate(over="ignore"):
        ref = _np_product(x, xs, y, ys, "f16")  # numpy half multiply: exact in f32, one rounding
    assert got.tobytes() == ref.view(np.uint16).tobytes()


def test_product_bf16_against_torch_and_tiny_values(orc):
    xs, ys = (4, 6, 5), (5, 5, 7)
    rng = np.random.default_rng(6)
    x = torch.from_numpy(rng.standard_normal(int(np.prod(xs))) * 100).to(torch.float32).to(torch.bfloat16)
    y = torch.from_numpy(rng.standard_normal(int(np.prod(ys)))).to(torch.float32).to(torch.bfloat16)
    xb = x.view(torch.int16).numpy().view(np.uint16)
    yb = y.view(torch.int16).numpy().view(np.uint16)
    got = orc.product(xb, xs, yb, ys, "bf16")
    I = tuple(min(a, b) for a, b in zip(xs, ys))
    sl = tuple(slice(0, s) for s in I)
    yy = y.reshape(ys).clone()
    # torch's bf16 multiply = exact f32 product + one rounding, valid in f32's normal range
    yy[sl] = (yy[sl].float() * x.reshape(xs)[sl].float()).to(torch.bfloat16)
    assert got.tobytes() == yy.reshape(-1).view(torch.int16).numpy().tobytes()
    # products below f32's normal range: compare with the brute-force nearest bf16
    bits, vals = _all_bf16_finite()
    for a, b in [(1e-20, 1e-20), (2.0 ** -70, 2.0 ** -64), (3e-39, 0.75), (2.0 ** -67 * 1.5, 2.0 ** -67 * 1.25)]:
        ab = orc.round_to(a, "bf16")
        bb = orc.round_to(b, "bf16")
        out = orc.product(np.array([ab], np.uint16), (1,), np.array([bb], np.uint16), (1,), "bf16")
        exact = orc.format_to_double(ab, "bf16") * orc.format_to_double(bb, "bf16")
        assert int(out[0]) == _bf16_brute(exact, bits, vals)


def test_product_properties_and_window(orc):
    xs, ys = (9, 9, 9, 9), (12, 8, 12, 8)
    rng = np.random.default_rng(8)
    y = rng.random(int(np.prod(ys)))
    ones = np.ones(int(np.prod(xs)))
    assert orc.product(ones, xs, y, ys, "f64").tobytes() == y.tobytes()
    x = rng.random(int(np.prod(xs)))
    full = orc.product(x, xs, y, ys, "f64", nthreads=3)
    assert full.tobytes() == orc.product(x, xs, y, ys, "f64", nthreads=1).tobytes()
    # outside the intersection nothing changes
    I = tuple(min(a, b) for a, b in zip(xs, ys))
    mask = np.ones(ys, dtype=bool)
    mask[tuple(slice(0, s) for s in I)] = False
    assert np.array_equal(full.reshape(ys)[mask], y.reshape(ys)[mask])
    for b, c in [(0, 100), (777, 5000), (full.size - 33, 33)]:
        w = orc.product_window(x, xs, y[b:b + c], ys, b, "f64")
        assert w.tobytes() == full[b:b + c].tobytes()
    # x == y (same shape) gives squares
    sq = orc.product(x, xs, x, xs, "f64")
    assert sq.tobytes() == (x * x).tobytes()


# ---------------------------------------------------------------- moment (Alg 10/11)

@pytest.mark.parametrize("shape", [(5,), (3, 4), (2, 3, 4), (4, 9, 7, 5), (2,) * 12])
def test_moment_point_mass_is_the_tuple(orc, shape):
    n = int(np.prod(shape))
    rng = np.random.default_rng(n)
    for k in [0, n - 1, int(rng.integers(0, n))]:
        p = np.zeros(n)
        p[k] = 1.0
        m = orc.moment(p, shape, "f64")
        t = np.unravel_index(k, shape)
        assert list(m[:-1]) == [float(v) for v in t] and m[-1] == 1.0


@pytest.mark.parametrize("shape", [(7,), (3, 4), (9, 9, 9), (2,) * 16, (5, 1, 6)])
def test_moment_constant_closed_form(orc, shape):
    n = int(np.prod(shape))
    m = orc.moment(np.ones(n), shape, "f64")
    expect = [n * (s - 1) / 2.0 for s in shape]  # integers: exact
    assert list(m[:-1]) == expect and m[-1] == float(n)


def test_moment_separable_closed_form(orc):
    shape = (6, 4, 7, 3)
    rng = np.random.default_rng(21)
    vs = [rng.random(s) for s in shape]
    p = vs[0]
    for v in vs[1:]:
        p = np.multiply.outer(p, v)
    m = orc.moment(p.reshape(-1), shape, "f64")
    sums = [v.sum() for v in vs]
    for i, v in enumerate(vs):
        expect = float(np.dot(np.arange(len(v)), v)) * float(np.prod([sums[j] for j in range(4) if j != i]))
        assert m[i] == pytest.approx(expect, rel=1e-13)
    assert m[-1] == pytest.approx(float(np.prod(sums)), rel=1e-13)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
def test_moment_brute_force_indices(orc, dtype):
    shape = (3, 5, 2, 4)
    rng = np.random.default_rng(22)
    v = rng.standard_normal(int(np.prod(shape)))
    if dtype == "f64":
        p = v
    elif dtype == "f32":
        p = v.astype(np.float32)
    else:
        p = orc.from_f64(v, dtype)
    w = orc.to_f64(p, dtype).reshape(shape)
    ind = np.indices(shape)
    m = orc.moment(p, shape, dtype)
    for i in range(len(shape)):
        assert m[i] == pytest.approx(float(np.sum(w * ind[i])), rel=1e-13, abs=1e-13)
    assert m[-1] == pytest.approx(float(np.sum(w)), rel=1e-13, abs=1e-13)


def test_moment_threads_match(orc):
    shape = (9, 9, 9, 9, 9)
    p = np.random.default_rng(23).random(int(np.prod(shape)))
    m1 = orc.moment(p, shape, "f64", nthreads=1)
    m5 = orc.moment(p, shape, "f64", nthreads=5)
    assert np.allclose(m1, m5, rtol=1e-15, atol=0)


@pytest.mark.parametrize("nthreads", [1, 3])
def test_moment_nonfinite_is_the_plain_ieee_sum(orc, nthreads):
    """A non-finite weight gives what the plain f64 sum of p[t] * t_i gives (IEEE rules)."""
    shape = (3, 4)
    base = np.random.default_rng(25).random(12)
    cases = [
        ({(1, 2): np.inf}, [np.inf, np.inf, np.inf]),
        ({(0, 2): np.inf}, [np.nan, np.inf, np.inf]),          # 0 * inf = NaN on axis 0
        ({(2, 3): -np.inf}, [-np.inf, -np.inf, -np.inf]),
        ({(1, 1): np.inf, (2, 2): -np.inf}, [np.nan, np.nan, np.nan]),
        ({(1, 3): np.nan}, [np.nan, np.nan, np.nan]),
    ]
    for bad, want in cases:
        p = base.copy().reshape(shape)
        for t, v in bad.items():
            p[t] = v
        got = orc.moment(p.reshape(-1), shape, "f64", nthreads=nthreads)
        for g_, w_ in zip(got, want):
            assert (np.isnan(g_) and np.isnan(w_)) or g_ == w_, (bad, got)


# ---------------------------------------------------------------- benchmark 3: x <- x + y x - z

APPLY_CASES = [((3, 4), (5, 7), (4, 9)), ((2, 3, 4), (2, 3, 4), (3, 5, 6)), ((5,), (9,), (5,)),
               ((3, 2, 2, 2), (4, 3, 5, 7), (8, 2, 6, 3))]


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("case", range(len(APPLY_CASES)))
def test_apply_xpyxmz_against_numpy(orc, dtype, case):
    xs, ys, zs = APPLY_CASES[case]
    rng = np.random.default_rng(95 + case)
    vals = [rng.standard_normal(int(np.prod(s))) for s in (xs, ys, zs)]
    if dtype != "f64":
        vals = [orc.from_f64(v, dtype) for v in vals]
    x, y, z = vals
    got = orc.apply_xpyxmz(x, xs, y, ys, z, zs, dtype)
    sl = tuple(slice(0, e) for e in xs)
    if dtype in ("f64", "f32"):
        ft = np.float64 if dtype == "f64" else np.float32
        X = x.reshape(xs).astype(ft)
        Y = y.reshape(ys)[sl].astype(ft)
        Z = z.reshape(zs)[sl].astype(ft)
        want = np.subtract(np.add(X, np.multiply(Y, X)), Z)
        assert got.tobytes() == want.astype(ft).tobytes()
    else:
        X = orc.to_f64(x, dtype).reshape(xs).astype(np.float32)
        Y = orc.to_f64(y, dtype).reshape(ys)[sl].astype(np.float32)
        Z = orc.to_f64(z, dtype).reshape(zs)[sl].astype(np.float32)
        r = np.subtract(np.add(X, np.multiply(Y, X)), Z)
        if dtype == "f16":
            want = r.astype(np.float16).view(np.uint16)
        else:
            want = torch.from_numpy(np.ascontiguousarray(r)).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
        assert got.tobytes() == np.ascontiguousarray(want).tobytes()


def test_apply_xpyxmz_special_cases(orc):
    xs, ys = (3, 4), (5, 6)
    x = np.random.default_rng(99).standard_normal(12)
    zero_y, zero_z = np.zeros(30), np.zeros(30)
    assert orc.apply_xpyxmz(x, xs, zero_y, ys, zero_z, ys, "f64").tobytes() == x.tobytes()  # x unchanged
    ones = np.ones(30)
    got = orc.apply_xpyxmz(x, xs, ones, ys, ones, ys, "f64")
    assert got.tobytes() == ((x + x) - 1.0).tobytes()                                       # 2x - 1


# ---------------------------------------------------------------- views (Section 4 bias)

VIEW_CASES = [((2, 3), (5, 7), (1, 4)), ((3, 1, 4), (6, 2, 9), (2, 1, 5)), ((4,), (4,), (0,)),
              ((2, 2, 2, 2), (3, 5, 2, 4), (1, 3, 0, 2)), ((0, 3), (4, 5), (2, 1))]


def _slices(st, xs):
    return tuple(slice(a, a + b) for a, b in zip(st, xs))


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("case", range(len(VIEW_CASES)))
def test_views_against_numpy_slicing(orc, dtype, case):
    xs, ys, st = VIEW_CASES[case]
    rng = np.random.default_rng(80 + case)
    x = orc.from_f64(rng.standard_normal(int(np.prod(xs))), dtype) if dtype != "f64" else rng.standard_normal(int(np.prod(xs)))
    y0 = orc.from_f64(rng.standard_normal(int(np.prod(ys))), dtype) if dtype != "f64" else rng.standard_normal(int(np.prod(ys)))
    # embed at: the window holds x, every other element is +0 (all bits zero)
    want = np.zeros(ys, dtype=x.dtype)
    want[_slices(st, xs)] = x.reshape(xs)
    assert orc.embed_at(x, xs, ys, st, dtype).tobytes() == want.tobytes()
    # NOPAD: the rest of y keeps its values
    want2 = y0.reshape(ys).copy()
    want2[_slices(st, xs)] = x.reshape(xs)
    assert orc.embed_at(x, xs, ys, st, dtype, y=y0).tobytes() == want2.tobytes()
    # crop at is the window read back; crop_at(embed_at(x)) = x
    assert orc.crop_at(y0, xs, ys, st, dtype).tobytes() == np.ascontiguousarray(y0.reshape(ys)[_slices(st, xs)]).tobytes()
    assert orc.crop_at(orc.embed_at(x, xs, ys, st, dtype), xs, ys, st, dtype).tobytes() == x.tobytes()


def test_product_at_against_numpy(orc):
    xs, ys, st = (4, 6, 3), (5, 8, 4), (2, 3, 2)     # x overhangs y on every axis
    rng = np.random.default_rng(90)
    x, y = rng.standard_normal(int(np.prod(xs))), rng.standard_normal(int(np.prod(ys)))
    got = orc.product_at(x, xs, y, ys, st, "f64").reshape(ys)
    fit = tuple(min(a, b - s) for a, b, s in zip(xs, ys, st))
    want = y.reshape(ys).copy()
    want[_slices(st, fit)] *= x.reshape(xs)[tuple(slice(0, f) for f in fit)]
    assert got.tobytes() == want.tobytes()


def test_bias_is_linear_in_the_tuple(orc):
    """Section 4's slice rule: idx(start + t) = idx(start) + idx(t) for in-bounds tuples."""
    shape = (4, 3, 5, 2)
    for start in [(0, 0, 0, 0), (1, 2, 3, 1), (3, 0, 4, 1)]:
        room = [s - a for s, a in zip(shape, start)]
        for t in itertools.product(*[range(r) for r in room]):
            s_t = [a + b for a, b in zip(start, t)]
            assert orc.tuple_to_index(s_t, shape) == orc.tuple_to_index(list(start), shape) + orc.tuple_to_index(list(t), shape)


# ---------------------------------------------------------------- moment of a product (Alg 11, n-ary)

MP_CASES = [
    [(3, 4), (5, 2)],
    [(2, 3, 4), (2, 3, 4)],
    [(4, 1, 3), (2, 5, 3), (3, 2, 2)],
    [(2, 2, 2, 2), (3, 1, 2, 5), (2, 2, 1, 2), (2, 3, 2, 2)],
    [(7,)],
    [(1, 1, 3), (2, 2, 2)],
]


def _brute_product_moment(xs, shapes, ftype):
    """numpy brute force: w over I (left-to-right products in ftype), exact f64 sums."""
    import math
    I = tuple(min(s[i] for s in shapes) for i in range(len(shapes[0])))
    sl = tuple(slice(0, e) for e in I)
    w = np.asarray(xs[0], dtype=np.float64).reshape(shapes[0])[sl].astype(ftype)
    for x, s in zip(xs[1:], shapes[1:]):
        w = (w * np.asarray(x, dtype=np.float64).reshape(s)[sl].astype(ftype)).astype(ftype)
    w = w.astype(np.float64)
    idx = np.indices(I) if len(I) else np.zeros((0,))
    m = [math.fsum((w * idx[i]).ravel()) for i in range(len(I))]
    return np.array(m + [math.fsum(w.ravel())])


@pytest.mark.parametrize("case", range(len(MP_CASES)))
def test_moment_product_brute_force_f64(orc, case):
    shapes = MP_CASES[case]
    rng = np.random.default_rng(40 + case)
    xs = [rng.standard_normal(int(np.prod(s))) for s in shapes]
    got = orc.moment_product(xs, shapes, "f64")
    want = _brute_product_moment(xs, shapes, np.float64)
    assert np.allclose(got, want, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_moment_product_float_products(orc, dtype):
    """Sub-f64 tensors: w is the float32 product chain of the exactly decoded values."""
    shapes = [(3, 5, 4), (4, 3, 6), (3, 4, 5)]
    rng = np.random.default_rng(50)
    xs = [orc.from_f64(rng.random(int(np.prod(s))) + 0.5, dtype) for s in shapes]
    dec = [orc.to_f64(x, dtype) for x in xs]
    got = orc.moment_product(xs, shapes, dtype)
    want = _brute_product_moment(dec, shapes, np.float32)
    assert np.allclose(got, want, rtol=1e-14, atol=0)


def test_moment_product_inner_product(orc):
    """Two tensors: the mass is the inner product over the tuples both shapes share."""
    xs_shape, ys_shape = (6, 7, 5), (4, 9, 5)
    rng = np.random.default_rng(51)
    x = rng.random(int(np.prod(xs_shape)))
    y = rng.random(int(np.prod(ys_shape)))
    got = orc.moment_product([x, y], [xs_shape, ys_shape], "f64")
    xa = x.reshape(xs_shape)[:4, :7, :5].ravel()
    ya = y.reshape(ys_shape)[:4, :7, :5].ravel()
    assert got[-1] == pytest.approx(float(np.dot(xa, ya)), rel=1e-14)


def test_moment_product_ones_closed_form(orc):
    """All-ones tensors: w = 1 on I, m_i = |I| (I_i - 1) / 2 exactly, mass |I|."""
    shapes = [(5, 6, 3, 4), (7, 4, 3, 9), (5, 5, 8, 4)]
    I = (5, 4, 3, 4)
    xs = [np.ones(int(np.prod(s))) for s in shapes]
    got = orc.moment_product(xs, shapes, "f64")
    n = int(np.prod(I))
    assert list(got) == [n * (e - 1) / 2 for e in I] + [float(n)]


def test_moment_product_separable_closed_form(orc):
    """x = a (x) b and y = c (x) d: w = (a c) (x) (b d) on I, so the moment factorises."""
    rng = np.random.default_rng(52)
    a, b, c, d = rng.random(6), rng.random(4), rng.random(5), rng.random(7)
    x = np.outer(a, b).ravel()
    y = np.outer(c, d).ravel()
    got = orc.moment_product([x, y], [(6, 4), (5, 7)], "f64")
    u, v = a[:5] * c, b[:4] * d[:4]
    want = [np.sum(np.arange(5) * u) * v.sum(), u.sum() * np.sum(np.arange(4) * v), u.sum() * v.sum()]
    assert np.allclose(got, want, rtol=1e-14)


def test_moment_product_single_tensor_is_the_moment(orc):
    shape = (4, 3, 5)
    p = np.random.default_rng(53).random(60)
    assert np.allclose(orc.moment_product([p], [shape], "f64"), orc.moment(p, shape, "f64"), rtol=1e-15)


# ---------------------------------------------------------------- convolution (Alg 14)

def test_convolution_against_scipy(orc):
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(24)
    a, b = rng.random((2 ** 5, 2 ** 3)), rng.random((2 ** 4, 2 ** 3))
    got = orc.convolve_f64(a, a.shape, b, b.shape)
    assert np.allclose(got, signal.convolve(a, b, method="direct"), rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------- Section 2: nonzero bounding box

def _bbox_numpy(tensors, shapes):
    """Brute force: the indices of the nonzero entries of the factors' product over the
    intersection, via numpy.nonzero (every factor nonzero)."""
    I = tuple(min(s[i] for s in shapes) for i in range(len(shapes[0])))
    nz = np.ones(I, dtype=bool)
    for x, s in zip(tensors, shapes):
        nz &= (x.reshape(s)[tuple(slice(0, e) for e in I)] != 0)
    idx = np.nonzero(nz)
    out = []
    for a in idx:
        out += [int(a.min()), int(a.max())] if a.size else [0, -1]
    return out + [int(nz.sum())]


@pytest.mark.parametrize("seed", range(6))
def test_nonzero_bbox_brute_force(orc, seed):
    rng = np.random.default_rng(400 + seed)
    d = int(rng.integers(1, 5))
    n = int(rng.integers(1, 4))
    shapes = [tuple(int(v) for v in rng.integers(1, 7, size=d)) for _ in range(n)]
    tensors = []
    for s in shapes:
        x = rng.standard_normal(int(np.prod(s)))
        x[rng.random(x.size) < 0.8] = 0.0         # mostly zero: boxes of all sizes
        tensors.append(x)
    assert list(orc.nonzero_bbox(tensors, shapes, "f64")) == _bbox_numpy(tensors, shapes)


def test_nonzero_bbox_closed_forms(orc):
    # a box-supported x times an all-ones y: the box clipped to the intersection
    xs, ys = (9, 8, 7), (6, 10, 7)
    x = np.zeros(xs)
    x[2:8, 3:5, 1:7] = 1.5
    y = np.ones(int(np.prod(ys)))
    got = orc.nonzero_bbox([x.reshape(-1), y], [xs, ys], "f64")
    assert list(got) == [2, 5, 3, 4, 1, 6, (6 - 2) * 2 * 6]
    # two boxes: their intersection; disjoint boxes: empty
    y2 = np.zeros(ys)
    y2[4:6, 0:4, 0:3] = -2.0
    assert list(orc.nonzero_bbox([x.reshape(-1), y2.reshape(-1)], [xs, ys], "f64")) == [4, 5, 3, 3, 1, 2, 2 * 1 * 2]
    y3 = np.zeros(ys)
    y3[0:2] = 1.0
    assert list(orc.nonzero_bbox([x.reshape(-1), y3.reshape(-1)], [xs, ys], "f64")) == [0, -1] * 3 + [0]
    # signed zeros never count; NaN and inf do; an empty intersection is empty
    z = np.array([0.0, -0.0, np.nan, np.inf, -0.0])
    assert list(orc.nonzero_bbox([z], [(5,)], "f64")) == [2, 3, 2]
    assert list(orc.nonzero_bbox([np.ones(6), np.ones(0)], [(2, 3), (0, 3)], "f64")) == [0, -1, 0, -1, 0]


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_nonzero_bbox_storage_types(orc, dtype):
    rng = np.random.default_rng(9)
    s1, s2 = (5, 6, 7), (6, 4, 8)
    a = rng.standard_normal(int(np.prod(s1)))
    b = rng.standard_normal(int(np.prod(s2)))
    a[rng.random(a.size) < 0.7] = 0.0
    b[rng.random(b.size) < 0.5] = -0.0
    # tiny values stay nonzero in storage; products that would underflow still count
    b[3] = 1e-30 if dtype != "f16" else 6e-8
    conv = (lambda v: v.astype(np.float32)) if dtype == "f32" else (lambda v: orc.from_f64(v, dtype))
    ra, rb = conv(a), conv(b)
    want = _bbox_numpy([orc.to_f64(ra, dtype), orc.to_f64(rb, dtype)], [s1, s2])
    assert list(orc.nonzero_bbox([ra, rb], [s1, s2], dtype)) == want


# ---------------------------------------------------------------- Section 4: windows on both sides

@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("seed", range(4))
def test_windows_both_sides_against_numpy_slicing(orc, dtype, seed):
    rng = np.random.default_rng(500 + seed)
    d = int(rng.integers(1, 5))
    ext = [int(v) for v in rng.integers(0, 5, size=d)]
    xs = [e + int(rng.integers(0, 4)) for e in ext]
    ys = [e + int(rng.integers(0, 4)) for e in ext]
    xo = [int(rng.integers(0, a - e + 1)) for a, e in zip(xs, ext)]
    yo = [int(rng.integers(0, a - e + 1)) for a, e in zip(ys, ext)]
    nx, ny = int(np.prod(xs)), int(np.prod(ys))
    xv = rng.standard_normal(nx) + 2.0
    yv = rng.standard_normal(ny) + 2.0
    if dtype == "f64":
        x, y = xv, yv
    elif dtype == "f32":
        x, y = xv.astype(np.float32), yv.astype(np.float32)
    else:
        x, y = orc.from_f64(xv, dtype), orc.from_f64(yv, dtype)
    xw = tuple(slice(o, o + e) for o, e in zip(xo, ext))
    yw = tuple(slice(o, o + e) for o, e in zip(yo, ext))
    want = y.reshape(ys).copy()
    want[yw] = x.reshape(xs)[xw]
    got = orc.copy_views(ext, x, xs, xo, y, ys, yo, dtype)
    assert got.tobytes() == want.reshape(-1).tobytes()
    # product: numpy elementwise on f64/f32, the oracle's own scalar product elsewhere
    got = orc.product_views(ext, x, xs, xo, y, ys, yo, dtype)
    if dtype in ("f64", "f32"):
        want = y.reshape(ys).copy()
        want[yw] = want[yw] * x.reshape(xs)[xw]
        assert got.tobytes() == want.reshape(-1).tobytes()
    else:
        sub = orc.product(x.reshape(xs)[xw].reshape(-1).copy(), ext, y.reshape(ys)[yw].reshape(-1).copy(), ext, dtype)
        want = y.reshape(ys).copy()
        want[yw] = sub.reshape(ext)
        assert got.tobytes() == want.reshape(-1).tobytes()


def test_windows_reduce_to_one_sided_views(orc):
    # x's window at the origin with x's full extent is product_at / crop_at
    xs, ys, st = (3, 4, 5), (6, 7, 9), (2, 1, 3)
    x = synth_like(int(np.prod(xs)), 31)
    y = synth_like(int(np.prod(ys)), 32)
    assert orc.product_views(xs, x, xs, (0, 0, 0), y, ys, st, "f64").tobytes() == \
        orc.product_at(x, xs, y, ys, st, "f64").tobytes()
    x2 = orc.copy_views(xs, y, ys, st, np.zeros(int(np.prod(xs))), xs, (0, 0, 0), "f64")
    assert x2.tobytes() == orc.crop_at(y, xs, ys, st, "f64").tobytes()


def synth_like(n, seed):
    return np.random.default_rng(seed).standard_normal(n)
