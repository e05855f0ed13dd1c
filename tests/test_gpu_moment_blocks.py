"""f64 moment on tensors whose trailing axes form blocks of at most 16 elements.

These shapes take the block-column fixed-point kernel: every block size B = 1..16, one to
sixteen outer axes (carries through several levels), tails that end inside a segment,
signed, subnormal, non-finite and unaligned input, and magnitudes that grow along the
segment (the segment exponent moves up while the sums are held).  The reference is the
oracle's compensated f64 sum (Algorithms 10 and 11); the tolerance is 1e-12 of
sum |p[t]| t_i per component.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1608_00099_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def tr():
    from paper_1608_00099_gb300 import build, triot
    build.build()
    triot.lib()
    assert torch.cuda.is_available()
    return triot


def scale(v, shape):
    return np.abs(orc.moment(np.abs(v), shape, "f64"))


def check(got, ref, sc):
    err = np.abs(got - ref)
    assert np.all(err <= TOL * sc + 1e-300), (got, ref, err / np.maximum(sc, 1e-300))


BLOCK_SHAPES = [
    (5,), (16,), (2, 2, 2, 2), (3, 7), (1000, 9), (7, 11, 13), (50, 3, 5), (33, 40, 2, 2, 3),
    (9,) * 6, (17, 19, 23, 14), (4,) * 10, (2,) * 20, (101, 103, 6), (5, 7, 9, 11, 2),
    (3,) * 12, (100003, 10), (31, 37, 41, 8), (3, 5, 7, 4), (2, 3, 1, 5, 1, 3), (61, 67, 11),
    (1, 1, 12), (8191, 1, 1),
]


@pytest.mark.parametrize("law", ["uniform", "normal"])
@pytest.mark.parametrize("shape", BLOCK_SHAPES)
def test_block_moment_matches_oracle(tr, shape, law):
    n = int(np.prod(shape))
    v = synth.uniform01(400 + n % 997, n) if law == "uniform" else synth.normal01(500 + n % 991, n)
    ref = orc.moment(v, shape, "f64")
    got = tr.triot_moment(torch.from_numpy(v.reshape(shape)).cuda()).cpu().numpy()
    check(got, ref, scale(v, shape))


@pytest.mark.parametrize("shape", [(40, 31, 16), (200, 300, 9), (7, 5, 3, 3, 4, 3)])
def test_block_moment_wide_range_subnormals_zeros(tr, shape):
    n = int(np.prod(shape))
    rng = np.random.default_rng(n)
    v = rng.standard_normal(n) * 10.0 ** rng.integers(-300, 300, size=n)
    v[:50] = rng.standard_normal(50) * 1e-310
    v[50:70] = 0.0
    v[70:80] = -0.0
    ref = orc.moment(v, shape, "f64")
    got = tr.triot_moment(torch.from_numpy(v.reshape(shape)).cuda()).cpu().numpy()
    check(got, ref, scale(v, shape))


@pytest.mark.parametrize("period,step", [(97, 1), (150, 3), (40, 7)])
def test_block_moment_growing_magnitudes(tr, period, step):
    shape = (300, 41, 9)
    n = int(np.prod(shape))
    k = np.arange(n)
    v = synth.uniform01(71, n) * np.exp2(((k * step) % period).astype(np.float64))
    ref = orc.moment(v, shape, "f64")
    got = tr.triot_moment(torch.from_numpy(v.reshape(shape)).cuda()).cpu().numpy()
    check(got, ref, scale(v, shape))


def test_block_moment_all_subnormal(tr):
    shape = (64, 33, 5)
    n = int(np.prod(shape))
    v = synth.uniform01(72, n) * 2.0 ** -1030
    ref = orc.moment(v, shape, "f64")
    got = tr.triot_moment(torch.from_numpy(v.reshape(shape)).cuda()).cpu().numpy()
    check(got, ref, scale(v, shape))


@pytest.mark.parametrize("bad", [np.inf, -np.inf, np.nan])
def test_block_moment_nonfinite(tr, bad):
    shape = (20, 30, 9)
    n = int(np.prod(shape))
    v = synth.uniform01(73, n)
    k = 3 * 270 + 5 * 9 + 4          # tuple (3, 5, 4): every component of the tuple is nonzero
    v[k] = bad
    got = tr.triot_moment(torch.from_numpy(v.reshape(shape)).cuda()).cpu().numpy()
    ref = orc.moment(v, shape, "f64")
    for g_, r_ in zip(got, ref):
        assert (np.isnan(g_) and np.isnan(r_)) or g_ == r_


def test_block_moment_unaligned(tr):
    shape = (37, 29, 3)
    n = int(np.prod(shape))
    v = synth.uniform01(74, n)
    buf = torch.empty(n + 8, dtype=torch.float64, device="cuda")
    p = buf[1:1 + n].view(shape)
    p.copy_(torch.from_numpy(v.reshape(shape)))
    got = tr.triot_moment(p).cpu().numpy()
    check(got, orc.moment(v, shape, "f64"), scale(v, shape))


def test_block_moment_point_masses(tr):
    shape = (13, 11, 7, 5, 3)
    n = int(np.prod(shape))
    for k in [0, 1, 14, 2 * 1155 + 17, n - 1]:
        p = torch.zeros(shape, dtype=torch.float64, device="cuda")
        p.view(-1)[k] = 0.75
        got = tr.triot_moment(p).cpu().numpy()
        assert list(got) == [0.75 * float(i) for i in np.unravel_index(k, shape)] + [0.75]
