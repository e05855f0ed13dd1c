"""The nonzero bounding box of a product of tensors (Section 2) against the oracle, bit for
bit (min / max / count are exact): one to four factors, every dtype, several tiles and
ragged rows, unit axes, long rows, sparse and dense supports, signed zeros, NaN and
infinities, empty results and an empty intersection."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1608_00099_gb300 import synth

from test_gpu_parity import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tr():
    from paper_1608_00099_gb300 import build, triot
    build.build()
    triot.lib()
    return triot


CASES = [
    [(9, 9, 9, 9), (12, 8, 12, 8)],
    [(5, 7)],
    [(3000,), (2999,)],
    [(6, 1, 5, 33), (4, 3, 7, 40), (5, 2, 6, 35)],
    [(2,) * 12, (3,) * 8 + (2,) * 4],
    [(2, 50000), (3, 40000)],
    [(17, 33, 65), (17, 40, 65), (20, 33, 70), (17, 35, 66)],
    [(1, 1, 4), (1, 2, 4)],
]


def _values(shape, dtype, seed, density):
    n = int(np.prod(shape))
    v = synth.normal01(seed, n)
    u = synth.uniform01(seed + 1, n)
    v[u >= density] = 0.0
    return v if dtype == "f64" else v.astype(np.float32) if dtype == "f32" else orc.from_f64(v, dtype)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("density", [1.0, 0.3, 0.001])
def test_bbox_against_oracle(tr, dtype, case, density):
    shapes = CASES[case]
    hs = [_values(s, dtype, 700 + 13 * k + case, density) for k, s in enumerate(shapes)]
    ref = orc.nonzero_bbox(hs, shapes, dtype)
    got = tr.triot_nonzero_bbox([to_dev(h, dtype, s) for h, s in zip(hs, shapes)]).cpu().numpy()
    assert list(got) == list(ref)


def test_bbox_box_support_and_specials(tr):
    xs, ys = (40, 30, 50), (35, 45, 48)
    x = torch.zeros(xs, dtype=torch.float64, device="cuda")
    x[7:31, 4:25, 9:44] = 1.0
    y = torch.ones(ys, dtype=torch.float64, device="cuda")
    y[:, :, 40:] = -0.0                                  # signed zeros do not count
    got = tr.triot_nonzero_bbox([x, y]).cpu().numpy()
    assert list(got) == [7, 30, 4, 24, 9, 39, (31 - 7) * (25 - 4) * (40 - 9)]
    z = torch.zeros(1000, dtype=torch.float32, device="cuda")
    z[[17, 912]] = torch.tensor([float("nan"), float("inf")], device="cuda")
    assert list(tr.triot_nonzero_bbox([z]).cpu().numpy()) == [17, 912, 2]
    e = torch.zeros((4, 0, 3), dtype=torch.float16, device="cuda")
    assert list(tr.triot_nonzero_bbox([e]).cpu().numpy()) == [0, -1] * 3 + [0]
    assert list(tr.triot_nonzero_bbox([torch.zeros((9, 8), device="cuda")]).cpu().numpy()) == [0, -1, 0, -1, 0]
    one = torch.full((1, 1), 2.0, device="cuda")
    assert list(tr.triot_nonzero_bbox([one]).cpu().numpy()) == [0, 0, 0, 0, 1]


def test_bbox_full_size_f64_d8_pair(tr):
    """The f64 d=8 pair (x 9^8, y (12,8)x4) with a sparse y: bit-exact at full size."""
    c8 = synth.config_f64_d8()
    xh = c8.x_values()
    yh = c8.yprod_values()
    yh[synth.uniform01(4242, yh.size) < 0.999] = 0.0
    x = torch.from_numpy(xh.reshape(c8.xshape)).cuda()
    y = torch.from_numpy(yh.reshape(c8.prod_shape)).cuda()
    got = tr.triot_nonzero_bbox([x, y]).cpu().numpy()
    ref = orc.nonzero_bbox([xh, yh], [c8.xshape, c8.prod_shape], "f64")
    assert list(got) == list(ref)
    assert tr.triot_nonzero_bbox([x, y]).cpu().numpy().tobytes() == got.tobytes()
