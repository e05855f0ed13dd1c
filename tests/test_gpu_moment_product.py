"""Moment of a product of tensors over the intersection of their shapes (Alg 11 with several
weight tensors; with two tensors the mass is benchmark 2's inner product), against the oracle.

Shapes span several rounds of 32 rows with ragged tails, unit axes in the intersection (a
non-unit-stride row axis), rows longer than the 1024-element fixed-point window, one to four
tensors, every dtype, signed/subnormal/zero/non-finite weights, and the full-size f64 d=8
pair (x 9^8 with y (12,8)x4) the product step uses.  Tolerance: 1e-12 of sum |w| t_i for f64
tensors, 1e-11 for float products (the products themselves are formed identically).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1608_00099_gb300 import synth

pytestmark = pytest.mark.gpu

TORCH = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}
TOL = {"f64": 1e-12, "f32": 1e-11, "bf16": 1e-11, "f16": 1e-11}


@pytest.fixture(scope="module")
def tr():
    from paper_1608_00099_gb300 import build, triot
    build.build()
    triot.lib()
    assert torch.cuda.is_available()
    return triot


def values(n, dtype, seed, law="normal"):
    v = synth.normal01(seed, n) if law == "normal" else synth.uniform01(seed, n)
    return orc.from_f64(v, dtype) if dtype != "f64" else v


def dev(a, dtype, shape):
    t = torch.from_numpy(np.ascontiguousarray(a).reshape(shape).copy())
    if dtype in ("bf16", "f16"):
        t = t.view(torch.int16).view(TORCH[dtype])
    return t.cuda()


def scale(xs, shapes, dtype):
    """sum |w| t_i and sum |w| from the oracle on |x_k|."""
    ab = [np.abs(orc.to_f64(x, dtype)) if dtype != "f64" else np.abs(x) for x in xs]
    ab = [orc.from_f64(a, dtype) if dtype != "f64" else a for a in ab]
    return np.abs(orc.moment_product(ab, shapes, dtype))


def check(tr, xs, shapes, dtype):
    ref = orc.moment_product(xs, shapes, dtype)
    got = tr.triot_moment_product([dev(x, dtype, s) for x, s in zip(xs, shapes)]).cpu().numpy()
    sc = scale(xs, shapes, dtype)
    err = np.abs(got - ref)
    assert np.all(err <= TOL[dtype] * sc + 1e-300), (got, ref, err / np.maximum(sc, 1e-300))


CASES = [
    [(3, 4), (5, 2)],
    [(40, 31, 17), (37, 33, 15)],
    [(9,) * 6, (11, 8, 11, 8, 11, 8)],
    [(4, 1, 3), (2, 5, 3), (3, 2, 2)],
    [(2, 2, 2, 2, 3, 5), (3, 1, 2, 5, 3, 5), (2, 2, 1, 2, 3, 5), (2, 3, 2, 2, 3, 5)],
    [(7,)],
    [(100003,), (100000,)],
    [(3, 3000), (2, 2900)],               # rows longer than the window
    [(1000, 7, 1), (999, 9, 2)],          # unit axis last: strided row axis
    [(1, 1, 3), (2, 2, 2)],
    [(6, 4, 7, 3, 5, 3, 3, 3, 6, 3), (7, 4, 6, 3, 5, 4, 3, 3, 6, 4)],
]


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_moment_product_matches_oracle(tr, dtype, case):
    shapes = CASES[case]
    xs = [values(int(np.prod(s)), dtype, 600 + 10 * case + k) for k, s in enumerate(shapes)]
    check(tr, xs, shapes, dtype)


def test_moment_product_f64_d8_pair_full_size(tr):
    """The product step's pair: the inner product and moment of x 9^8 and y (12,8)x4."""
    xs_shape, ys_shape = (9,) * 8, (12, 8) * 4
    x = synth.uniform01(1002, 9 ** 8)
    y = synth.uniform01(1003, int(np.prod(ys_shape)))
    check(tr, [x, y], [xs_shape, ys_shape], "f64")


def test_moment_product_wide_range_and_specials(tr):
    rng = np.random.default_rng(61)
    shapes = [(50, 40, 9), (48, 41, 9)]
    xs = [rng.standard_normal(int(np.prod(s))) * 10.0 ** rng.integers(-150, 150, size=int(np.prod(s)))
          for s in shapes]
    xs[0][:30] = rng.standard_normal(30) * 1e-310
    xs[1][30:40] = 0.0
    check(tr, xs, shapes, "f64")
    xs[0][5 * 360 + 7 * 9 + 3] = np.inf   # tuple (5, 7, 3): every component nonzero
    got = tr.triot_moment_product([dev(x, "f64", s) for x, s in zip(xs, shapes)]).cpu().numpy()
    ref = orc.moment_product(xs, shapes, "f64")
    for g_, r_ in zip(got, ref):
        assert (np.isnan(g_) and np.isnan(r_)) or g_ == r_


def test_moment_product_empty_and_single(tr):
    z = tr.triot_moment_product([torch.ones((3, 0, 2), dtype=torch.float64, device="cuda"),
                                 torch.ones((3, 4, 2), dtype=torch.float64, device="cuda")]).cpu().numpy()
    assert list(z) == [0.0] * 4
    one = tr.triot_moment_product([torch.full((1, 1), 3.0, dtype=torch.float64, device="cuda"),
                                   torch.full((2, 2), 0.5, dtype=torch.float64, device="cuda")]).cpu().numpy()
    assert list(one) == [0.0, 0.0, 1.5]


def test_moment_product_point_mass_exact_and_deterministic(tr):
    shapes = [(13, 11, 7), (12, 12, 9)]
    for t in [(0, 0, 0), (4, 9, 2), (11, 10, 6)]:
        x = torch.zeros(shapes[0], dtype=torch.float64, device="cuda")
        y = torch.zeros(shapes[1], dtype=torch.float64, device="cuda")
        x[t] = 0.75
        y[t] = 2.0
        got = tr.triot_moment_product([x, y]).cpu().numpy()
        assert list(got) == [1.5 * v for v in t] + [1.5]
    xs = [values(int(np.prod(s)), "f64", 70 + k) for k, s in enumerate(shapes)]
    ts = [dev(x, "f64", s) for x, s in zip(xs, shapes)]
    a = tr.triot_moment_product(ts).cpu().numpy()
    b = tr.triot_moment_product(ts).cpu().numpy()
    assert a.tobytes() == b.tobytes()


# rows of I shorter than 8 elements take the tiled short-row kernel: several tiles and a
# partial last one, strided row axes, two to four factors, every dtype
SHORT = [
    [(300, 41, 2), (301, 40, 3)],
    [(9, 8, 9, 8, 9, 4), (9, 9, 9, 9, 9, 5)],
    [(64, 33, 7), (65, 32, 7), (64, 32, 8)],
    [(40, 1, 30, 5), (41, 3, 30, 6), (40, 2, 31, 5), (42, 1, 30, 5)],
    [(5000, 3, 1), (5001, 4, 2)],
]


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("case", range(len(SHORT)))
def test_moment_product_short_rows(tr, dtype, case):
    shapes = SHORT[case]
    xs = [values(int(np.prod(s)), dtype, 900 + 10 * case + k) for k, s in enumerate(shapes)]
    check(tr, xs, shapes, dtype)


@pytest.mark.parametrize("where", ["first", "last"])
def test_moment_product_short_rows_wide_range_and_specials(tr, where):
    rng = np.random.default_rng(62)
    shapes = [(60, 50, 3), (61, 50, 4)]
    xs = [rng.standard_normal(int(np.prod(s))) * 10.0 ** rng.integers(-150, 150, size=int(np.prod(s)))
          for s in shapes]
    xs[0][:40] = rng.standard_normal(40) * 1e-310
    xs[1][50:70] = 0.0
    check(tr, xs, shapes, "f64")
    t = (5, 7, 2) if where == "first" else (59, 49, 1)
    xs[0][t[0] * 150 + t[1] * 3 + t[2]] = np.inf
    xs[1][t[0] * 200 + t[1] * 4 + t[2]] = 2.0     # y at the same tuple: finite and nonzero
    if where == "last":
        xs[0][(t[0] // 2) * 150 + 3 * 3 + 0] = np.nan   # tuple (29, 3, 0), in another tile
    got = tr.triot_moment_product([dev(x, "f64", s) for x, s in zip(xs, shapes)]).cpu().numpy()
    ref = orc.moment_product(xs, shapes, "f64")
    for g_, r_ in zip(got, ref):
        assert (np.isnan(g_) and np.isnan(r_)) or g_ == r_, (got, ref)


def test_moment_product_short_rows_point_masses_exact(tr):
    shapes = [(33, 17, 5), (34, 17, 6)]
    for t in [(0, 0, 0), (32, 16, 4), (17, 3, 2)]:
        x = torch.zeros(shapes[0], dtype=torch.float32, device="cuda")
        y = torch.zeros(shapes[1], dtype=torch.float32, device="cuda")
        x[t] = 0.75
        y[t] = 2.0
        got = tr.triot_moment_product([x, y]).cpu().numpy()
        assert list(got) == [1.5 * v for v in t] + [1.5]
