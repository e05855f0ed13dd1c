"""Parity at the full workload sizes, in the launch configuration bench.py times.

The f64 d=8 step runs twice: under the default geometry and under the committed tuning
file that bench.py loads before it times the step (paper_1608_00099_gb300/tune_gb300.json).

Small and medium cases are compared in full; the 44 GB embed target of the f32 d=24
workload is compared on windows the oracle computes one element at a time, and through
properties that hold at any size (pad count, crop round trip).
"""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1608_00099_gb300 import synth

from test_gpu_parity import TORCH, check_moment, moment_scale, to_dev, to_host

pytestmark = pytest.mark.gpu
NT = min(16, os.cpu_count() or 1)


@pytest.fixture(scope="module")
def tr():
    from paper_1608_00099_gb300 import build, triot
    build.build()
    triot.lib()
    return triot


def test_embed_f64_d6_full(tr):
    cfg = synth.config_embed_small()
    xh = cfg.x_values()
    x = torch.from_numpy(xh.reshape(cfg.xshape)).cuda()
    y = torch.empty(cfg.embed_shape, dtype=torch.float64, device="cuda")
    tr.triot_embed(x, y)
    ref = orc.embed(xh, cfg.xshape, cfg.embed_shape, "f64")
    assert y.cpu().numpy().reshape(-1).tobytes() == ref.tobytes()
    x2 = torch.empty_like(x)
    tr.triot_crop(x2, y)
    assert torch.equal(x2, x)


TUNE_FILE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                         "paper_1608_00099_gb300", "tune_gb300.json")


@pytest.fixture(params=["default", "tuned"])
def geometry(request, tr):
    tr.triot_tune_clear()
    if request.param == "tuned":
        tr.triot_tune_load(TUNE_FILE)
    yield request.param
    tr.triot_tune_clear()


@pytest.fixture(scope="module")
def f64_d8():
    cfg = synth.config_f64_d8()
    xh = cfg.x_values()
    return cfg, xh


def test_f64_d8_embed_full(tr, f64_d8, geometry):
    cfg, xh = f64_d8
    x = torch.from_numpy(xh.reshape(cfg.xshape)).cuda()
    y = torch.empty(cfg.embed_shape, dtype=torch.float64, device="cuda")
    tr.triot_embed(x, y)
    ref = orc.embed(xh, cfg.xshape, cfg.embed_shape, "f64", nthreads=NT)
    assert np.array_equal(y.cpu().numpy().reshape(-1).view(np.uint64), ref.view(np.uint64))
    x2 = torch.empty_like(x)
    tr.triot_crop(x2, y)
    assert torch.equal(x2, x)


def test_f64_d8_product_full(tr, f64_d8, geometry):
    cfg, xh = f64_d8
    yh = cfg.yprod_values()
    x = torch.from_numpy(xh.reshape(cfg.xshape)).cuda()
    y = torch.from_numpy(yh.reshape(cfg.prod_shape)).cuda()
    tr.triot_product(x, y)
    ref = orc.product(xh, cfg.xshape, yh, cfg.prod_shape, "f64", nthreads=NT)
    assert np.array_equal(y.cpu().numpy().reshape(-1).view(np.uint64), ref.view(np.uint64))


def test_f64_d8_moment_full(tr, f64_d8, geometry):
    cfg, xh = f64_d8
    ph = synth.normalise(xh)
    p = torch.from_numpy(ph.reshape(cfg.xshape)).cuda()
    got = tr.triot_moment(p).cpu().numpy()
    ref = orc.moment(ph, cfg.xshape, "f64", nthreads=NT)
    check_moment(got, ref, np.abs(ref), 1e-12)   # p >= 0: the scale is the value itself
    again = tr.triot_moment(p).cpu().numpy()
    assert again.tobytes() == got.tobytes()


@pytest.mark.slow
def test_f32_d24_embed_product_moment_sampled(tr):
    cfg = synth.config_f32_d24()
    xh = cfg.x_values().astype(np.float32)
    ny = int(np.prod(cfg.embed_shape))
    free, _ = torch.cuda.mem_get_info()
    if free < ny * 4 + (4 << 30):
        pytest.skip("not enough device memory for the 44 GB target")
    x = torch.from_numpy(xh.reshape(cfg.xshape)).cuda()
    y = torch.empty(ny, dtype=torch.float32, device="cuda").view(cfg.embed_shape)
    y.view(-1)[:1 << 20].fill_(7.0)
    tr.triot_embed(x, y)
    rng = np.random.default_rng(99)
    w = 1 << 20
    starts = [0, ny - w] + [int(s) for s in rng.integers(0, ny - w, size=14)]
    yflat = y.view(-1)
    for s in starts:
        ref = orc.embed_window(xh, cfg.xshape, cfg.embed_shape, s, w, "f32")
        assert yflat[s:s + w].cpu().numpy().tobytes() == ref.tobytes(), s
    # property at full size: exactly |x| elements are nonzero (x has no zeros) ...
    assert int((xh == 0).sum()) == 0
    nz = int(torch.count_nonzero(yflat).item())
    assert nz == xh.size
    # ... and cropping gives x back
    x2 = torch.empty_like(x)
    tr.triot_crop(x2, y)
    assert torch.equal(x2, x)
    # product over the all-2 intersection: windows against the oracle
    tr.triot_product(x, y)
    for s in starts[:8]:
        before = orc.embed_window(xh, cfg.xshape, cfg.embed_shape, s, w, "f32")
        ref = orc.product_window(xh, cfg.xshape, before, cfg.embed_shape, s, "f32")
        assert yflat[s:s + w].cpu().numpy().tobytes() == ref.tobytes(), s
    x3 = torch.empty_like(x)
    tr.triot_crop(x3, y)
    assert np.array_equal(x3.cpu().numpy().reshape(-1), xh * xh)
    del y, yflat
    torch.cuda.empty_cache()
    got = tr.triot_moment(x).cpu().numpy()
    ref = orc.moment(xh, cfg.xshape, "f32", nthreads=NT)
    check_moment(got, ref, np.abs(ref), 1e-5)


@pytest.mark.parametrize("dtype", ["bf16", "f16", "f64"])
def test_precision_workload(tr, dtype):
    pc = synth.config_precision()
    I = tuple(min(a, b) for a, b in zip(pc.pshape, pc.qshape))
    ph = orc.from_f64(pc.p64, dtype)
    qh = orc.from_f64(pc.q64, dtype)
    p = to_dev(ph, dtype, pc.pshape)
    q = to_dev(qh, dtype, pc.qshape)
    r = torch.empty(I, dtype=TORCH[dtype], device="cuda")
    tr.triot_crop(r, p)
    tr.triot_product(q, r)
    m = tr.triot_moment(r).cpu().numpy()
    rh = orc.crop(ph, I, pc.pshape, dtype)
    rh = orc.product(qh, pc.qshape, rh, I, dtype)
    assert to_host(r, dtype).tobytes() == rh.tobytes()
    ref = orc.moment(rh, I, dtype)
    check_moment(m, ref, moment_scale(rh, I, dtype), 1e-12 if dtype == "f64" else 1e-5)
    # error of the rounded product against the exact product of the rounded inputs
    if dtype != "f64":
        exact = orc.to_f64(orc.crop(ph, I, pc.pshape, dtype), dtype) * orc.to_f64(orc.crop(qh, I, pc.qshape, dtype), dtype)
        got = orc.to_f64(to_host(r, dtype), dtype)
        normal = np.abs(exact) >= (2.0 ** -126 if dtype == "bf16" else 2.0 ** -14)
        rel = np.abs(got[normal] - exact[normal]) / np.abs(exact[normal])
        assert np.all(rel <= 2.0 ** -8)
        if dtype == "f16":
            assert np.all(np.abs(got[~normal] - exact[~normal]) <= 2.0 ** -25)


@pytest.mark.slow
@pytest.mark.parametrize("mode", ["fused", "plain"])
def test_batch_full(tr, mode):
    pairs = synth.config_batch_shapes()
    xs_h = synth.batch_x_values(pairs)
    xs, ys, outs = [], [], []
    for pr, xh in zip(pairs, xs_h):
        xs.append(torch.from_numpy(xh.astype(np.float32).reshape(pr.xshape)).cuda())
        ys.append(torch.empty(pr.yshape, dtype=torch.float32, device="cuda"))
        outs.append(torch.zeros(len(pr.xshape) + 1, dtype=torch.float64, device="cuda"))
    plan = tr.BatchPlan(xs, ys, outs, mode=tr.BATCH_FUSED)
    if mode == "plain":
        plan.run_plain()
    else:
        plan.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    check = sorted(set([0, len(pairs) - 1] + [int(i) for i in rng.integers(0, len(pairs), size=200)]))
    for k in check:
        pr = pairs[k]
        xh = xs_h[k].astype(np.float32)
        ye = orc.product(xh, pr.xshape, orc.embed(xh, pr.xshape, pr.yshape, "f32"), pr.yshape, "f32")
        assert ys[k].cpu().numpy().reshape(-1).tobytes() == ye.tobytes(), k
        ref = orc.moment(ye, pr.yshape, "f32")
        check_moment(outs[k].cpu().numpy(), ref, np.abs(ref), 1e-5)
    plan.close()
