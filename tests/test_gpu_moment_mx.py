"""The f64 moment by marginals (rows x columns split) against the oracle.

Shapes are chosen so that triot_moment_plan reports the marginal kernel, with splits of
one to many row axes (so the lazy carry of the row digits is exercised at every depth),
column tiles that are full and partial, rows per warp from one to several windows, and
values that leave the lean conversion: signed, subnormal, zero, wide exponent ranges,
growing magnitudes, non-finite.  Tolerance as every f64 moment: 1e-12 of sum |p| t_i.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1608_00099_gb300 import synth

from test_gpu_parity import check_moment, moment_scale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tr():
    from paper_1608_00099_gb300 import build, triot
    build.build()
    triot.lib()
    triot.triot_tune_clear()
    return triot


MX_SHAPES = [
    (9,) * 7,                    # 26 tiles of columns, the last partial
    (2,) * 22,                   # many row axes of extent 2: carries at every depth
    (5, 3, 7, 8, 4096),
    (7, 4, 3, 5, 2, 9, 400),
    (30, 100000),                # long rows, few of them
    (5000, 1, 500),              # a unit axis between rows and columns
    (6, 4, 7, 3, 5, 6, 7, 3, 7, 3),
    (110, 130, 256),
]


@pytest.mark.parametrize("shape", MX_SHAPES)
@pytest.mark.parametrize("law", ["uniform", "normal"])
def test_mx_moment_against_oracle(tr, shape, law):
    plan = tr.triot_moment_plan(shape, torch.float64)
    assert plan["kernel"] == "marginals", plan
    n = int(np.prod(shape))
    v = synth.uniform01(3100 + n, n) if law == "uniform" else synth.normal01(3100 + n, n)
    ref = orc.moment(v, shape, "f64")
    p = torch.from_numpy(v.reshape(shape)).cuda()
    got = tr.triot_moment(p).cpu().numpy()
    check_moment(got, ref, moment_scale(v, shape, "f64"), 1e-12)
    assert tr.triot_moment(p).cpu().numpy().tobytes() == got.tobytes()


@pytest.mark.parametrize("shape", [(9,) * 7, (2,) * 22, (5, 3, 7, 8, 4096)])
def test_mx_point_masses_exact(tr, shape):
    n = int(np.prod(shape))
    for k in [0, 1, n // 3, n - 1]:
        p = torch.zeros(shape, dtype=torch.float64, device="cuda")
        p.view(-1)[k] = 0.375
        m = tr.triot_moment(p).cpu().numpy()
        assert list(m) == [0.375 * float(t) for t in np.unravel_index(k, shape)] + [0.375]


@pytest.mark.parametrize("case", ["wide", "subnormal_zero", "growing", "signed_growing", "tiny_only"])
def test_mx_dynamic_range(tr, case):
    shape = (40, 31, 170, 16)
    n = int(np.prod(shape))
    seeds = {"wide": 1, "subnormal_zero": 2, "growing": 3, "signed_growing": 4, "tiny_only": 5}
    rng = np.random.default_rng(seeds[case])
    if case == "wide":
        v = rng.standard_normal(n) * 10.0 ** rng.integers(-300, 300, size=n)
    elif case == "subnormal_zero":
        v = rng.random(n)
        v[::7] = 0.0
        v[::11] = rng.random(len(v[::11])) * 1e-310
    elif case == "growing":
        v = rng.random(n) * np.exp(np.linspace(0, 200, n))        # every row raises the exponent
    elif case == "signed_growing":
        v = rng.standard_normal(n) * np.exp(np.linspace(0, 60, n))
    else:
        v = rng.random(n) * 1e-308                                # window exponents below 54
    assert tr.triot_moment_plan(shape, torch.float64)["kernel"] == "marginals"
    ref = orc.moment(v, shape, "f64")
    got = tr.triot_moment(torch.from_numpy(v.reshape(shape)).cuda()).cpu().numpy()
    check_moment(got, ref, moment_scale(v, shape, "f64"), 1e-12)


@pytest.mark.parametrize("where", ["first", "middle", "last_row", "partial_tile"])
def test_mx_nonfinite_against_oracle(tr, where):
    shape = (9,) * 7
    n = int(np.prod(shape))
    v = synth.uniform01(77, n) - 0.25
    k = {"first": 0, "middle": n // 2 + 13, "last_row": n - 100, "partial_tile": 9 ** 4 - 3}[where]
    v[k] = np.inf
    v[(k + 4000) % n] = -np.inf if where == "middle" else np.nan
    ref = orc.moment(v, shape, "f64")
    got = tr.triot_moment(torch.from_numpy(v.reshape(shape)).cuda()).cpu().numpy()
    for g, r in zip(got, ref):
        if np.isnan(r):
            assert np.isnan(g)
        else:
            assert g == r


def test_mx_many_windows_separable_closed_form(tr):
    """Rows per warp above one window (ctas_per_sm forced to 1): p = a[r] b[c] with small
    integer factors, whose moments are exact integers given by the marginals."""
    R, C = 1 << 21, 256
    shape = (R, C)
    tr.triot_tune_set(tr.OP_MOMENT, shape, None, torch.float64, ctas_per_sm=1)
    try:
        plan = tr.triot_moment_plan(shape, torch.float64)
        assert plan["kernel"] == "marginals" and plan["rows"] == R
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert R / (sms * 8) > 1023          # more than one window per warp
        a = (torch.arange(R, dtype=torch.float64, device="cuda") % 7) + 1
        b = (torch.arange(C, dtype=torch.float64, device="cuda") % 5) + 1
        p = a[:, None] * b[None, :]
        got = tr.triot_moment(p).cpu().numpy()
        ah, bh = a.cpu().numpy(), b.cpu().numpy()
        r_idx, c_idx = np.arange(R, dtype=np.float64), np.arange(C, dtype=np.float64)
        ref = [float((ah * r_idx).sum() * bh.sum()), float(ah.sum() * (bh * c_idx).sum()),
               float(ah.sum() * bh.sum())]
        assert list(got) == ref
    finally:
        tr.triot_tune_clear()


# float storage takes the marginal kernel for large tensors whose rows are 16-byte multiples
MX32_CASES = [
    ("f32", (4,) * 13, False),             # 67M elements, vector loads
    ("f32", (4,) * 13, True),              # the same from a pointer 4 bytes past a 16-byte bound
    ("bf16", (4,) * 12 + (2,), False),     # 33.5M elements, eight per vector
    ("f16", (8, 4096, 1024), False),
    ("bf16", (3, 5, 7, 320000), False),    # a partial last tile (320000 % 512 != 0)
]


@pytest.mark.slow
@pytest.mark.parametrize("dtype,shape,shifted", MX32_CASES)
def test_mx_float_moment_against_oracle(tr, dtype, shape, shifted):
    from test_gpu_parity import TORCH, host_values, misaligned, to_dev
    plan = tr.triot_moment_plan(shape, TORCH[dtype])
    assert plan["kernel"] == "marginals", plan
    n = int(np.prod(shape))
    ph = host_values(n, dtype, 4100 + len(shape), law="uniform")
    if shifted:
        p = misaligned(shape, dtype)
        p.copy_(to_dev(ph, dtype, shape))
    else:
        p = to_dev(ph, dtype, shape)
    got = tr.triot_moment(p).cpu().numpy()
    ref = orc.moment(ph, shape, dtype, nthreads=16)
    check_moment(got, ref, np.abs(ref), 1e-5)   # p >= 0: the scale is the value itself
    assert tr.triot_moment(p).cpu().numpy().tobytes() == got.tobytes()
