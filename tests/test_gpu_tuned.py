"""Parity under tuned launch geometries.

The autotuner (triot_autotune, triot_batch_autotune) picks tile sizes and CTAs per SM by
measurement; a geometry only changes how the work is split, never what is computed, and
these tests hold it to that: every op is rerun under the geometry the autotuner chose and
compared with the oracle (bit for bit; moments within their tolerance).
"""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1608_00099_gb300 import synth

from test_gpu_parity import check_moment, moment_scale

pytestmark = pytest.mark.gpu
NT = min(16, os.cpu_count() or 1)


@pytest.fixture()
def tr():
    from paper_1608_00099_gb300 import build, triot
    build.build()
    triot.lib()
    triot.triot_tune_clear()
    yield triot
    triot.triot_tune_clear()


# mid-size f64 shapes (about 40-120 MB per tensor): the f64 d=8 workload with one axis fewer
XS = (9,) * 7
EMB = (11, 10, 11, 10, 11, 10, 11)
PRD = (12, 8, 12, 8, 12, 8, 12)


def test_autotune_embed_then_parity(tr):
    xh = synth.uniform01(2201, int(np.prod(XS)))
    x = torch.from_numpy(xh.reshape(XS)).cuda()
    y = torch.empty(EMB, dtype=torch.float64, device="cuda")
    best = tr.triot_autotune(tr.OP_EMBED, x, y)
    assert best["tile_elems"] > 0 and best["ctas_per_sm"] > 0
    assert tr.triot_tune_get(tr.OP_EMBED, XS, EMB, torch.float64) == best
    y.fill_(7.0)
    tr.triot_embed(x, y)   # runs under the cached (tuned) geometry
    ref = orc.embed(xh, XS, EMB, "f64", nthreads=NT)
    assert np.array_equal(y.cpu().numpy().reshape(-1).view(np.uint64), ref.view(np.uint64))
    x2 = torch.empty_like(x)
    tr.triot_autotune(tr.OP_CROP, x2, y)
    x2.zero_()
    tr.triot_crop(x2, y)
    assert torch.equal(x2, x)


def test_autotune_product_then_parity(tr):
    xh = synth.uniform01(2202, int(np.prod(XS)))
    yh = synth.uniform01(2203, int(np.prod(PRD)))
    x = torch.from_numpy(xh.reshape(XS)).cuda()
    y = torch.from_numpy(yh.reshape(PRD)).cuda()
    best = tr.triot_autotune(tr.OP_PRODUCT, x, y)   # overwrites y many times
    assert best["tile_elems"] > 0
    y.copy_(torch.from_numpy(yh.reshape(PRD)))
    tr.triot_product(x, y)
    ref = orc.product(xh, XS, yh, PRD, "f64", nthreads=NT)
    assert np.array_equal(y.cpu().numpy().reshape(-1).view(np.uint64), ref.view(np.uint64))


@pytest.mark.parametrize("dtype,shape", [("f64", XS), ("f32", (2,) * 22), ("f32", (9, 9, 9, 9, 9, 9, 9))])
def test_autotune_moment_then_parity(tr, dtype, shape):
    n = int(np.prod(shape))
    ph = synth.normalise(synth.uniform01(2204, n))
    if dtype == "f32":
        ph = ph.astype(np.float32)
    p = torch.from_numpy(ph.reshape(shape)).cuda()
    best = tr.triot_autotune(tr.OP_MOMENT, p)
    assert best["ctas_per_sm"] > 0
    got = tr.triot_moment(p).cpu().numpy()
    ref = orc.moment(ph, shape, dtype, nthreads=NT)
    check_moment(got, ref, moment_scale(ph, shape, dtype), 1e-12 if dtype == "f64" else 1e-5)


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_autotune_then_parity(tr, mode):
    pairs = synth.config_batch_shapes()[:384]
    xs_h = synth.batch_x_values(pairs)
    xs, ys, outs = [], [], []
    for pr, xh in zip(pairs, xs_h):
        xs.append(torch.from_numpy(xh.astype(np.float32).reshape(pr.xshape)).cuda())
        ys.append(torch.empty(pr.yshape, dtype=torch.float32, device="cuda"))
        outs.append(torch.zeros(len(pr.xshape) + 1, dtype=torch.float64, device="cuda"))
    best = tr.triot_batch_autotune(xs, ys, outs, mode=mode)
    assert best["tile_elems"] in (256, 512, 1024, 2048, 4096) and best["ctas_per_sm"] in (2, 4, 8)
    plan = tr.BatchPlan(xs, ys, outs, mode=mode)   # zero tune fields: the cached geometry
    geo = plan.geometry()
    assert (geo["tile_elems"], geo["ctas_per_sm"]) == (best["tile_elems"], best["ctas_per_sm"])
    for y in ys:
        y.fill_(5.0)
    for o in outs:
        o.fill_(float("nan"))
    plan.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(17)
    for k in sorted(set([0, len(pairs) - 1] + [int(i) for i in rng.integers(0, len(pairs), size=60)])):
        pr = pairs[k]
        xh = xs_h[k].astype(np.float32)
        ye = orc.product(xh, pr.xshape, orc.embed(xh, pr.xshape, pr.yshape, "f32"), pr.yshape, "f32")
        assert ys[k].cpu().numpy().reshape(-1).tobytes() == ye.tobytes(), k
        ref = orc.moment(ye, pr.yshape, "f32")
        check_moment(outs[k].cpu().numpy(), ref, np.abs(ref), 1e-5)
    plan.close()
