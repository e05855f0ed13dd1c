"""Benchmark 3 of Section 3, x[t] <- x[t] + y[t] x[t] - z[t] over x's shape with y and z of
other (larger) shapes, bit for bit against the oracle for every dtype: the benchmark's own
shapes, multi-tile and long-row (segmented) cases, unit axes, merged axes, and empty x."""
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
    ((2 ** 7 + 1, 2 ** 5, 2 ** 3 + 5, 2 ** 4), (2 ** 8 - 3, 2 ** 6, 2 ** 6, 2 ** 4 + 7),
     (2 ** 8, 2 ** 5 + 7, 2 ** 6, 2 ** 5 + 1)),                       # benchmark 3's shapes
    ((3, 4), (5, 7), (4, 9)),
    ((5, 20000), (6, 20001), (5, 30000)),                           # segmented rows
    ((7, 1, 9, 1), (8, 3, 9, 2), (7, 2, 10, 1)),                    # unit axes
    ((4, 6, 8), (4, 6, 8), (4, 6, 8)),                              # one merged row
    ((0, 5), (2, 5), (3, 5)),                                       # empty x
]


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_apply_xpyxmz_bit_exact(tr, dtype, case):
    xs, ys, zs = CASES[case]
    xh = values(int(np.prod(xs)), dtype, 800 + case)
    yh = values(int(np.prod(ys)), dtype, 820 + case)
    zh = values(int(np.prod(zs)), dtype, 840 + case)
    x = dev(xh, dtype, xs)
    tr.triot_apply_xpyxmz(x, dev(yh, dtype, ys), dev(zh, dtype, zs))
    assert host(x, dtype).tobytes() == orc.apply_xpyxmz(xh, xs, yh, ys, zh, zs, dtype).tobytes()
