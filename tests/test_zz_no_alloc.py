"""The allocation-free moment entry point (triot_moment_noalloc).

Some callers cannot allocate device memory -- code running where cudaMalloc is forbidden or
would synchronise the device, or an application whose device memory is all handed out by its
own pool -- so they cannot hand triot_moment a workspace.  triot_moment_noalloc keeps its
partial sums in a fixed scratch array inside the library instead.  These tests call it
through the C ABI, compare it element by element with the CPU oracle (within the moment
tolerances the other tests use) and bit for bit with triot_moment (the same plan, kernels
and order-independent combine), over calls in a row on different data of one shape, since
the scratch keeps the previous call's contents.  The file is collected last.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1608_00099_gb300 import synth

from test_gpu_parity import TORCH, check_moment, host_values, moment_scale, to_dev

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 1e-5}


@pytest.fixture(scope="module")
def tr():
    from paper_1608_00099_gb300 import build, triot
    build.build()
    triot.lib()
    return triot


def _noalloc(tr, p, out):
    st = tr.lib().triot_moment_noalloc(p.dim(), tr._shape(p.shape), p.data_ptr(), tr._dtype(p),
                                       out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    if st != 0:
        raise tr.TriotError(st, tr.lib().triot_last_error().decode())
    return out


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("shape", [(9, 9, 9, 9, 9), (37, 1, 41), (2,) * 14])
def test_noalloc_matches_oracle_on_alternating_data(tr, dtype, shape):
    n = int(np.prod(shape))
    data = [host_values(n, dtype, 9100 + k, law="uniform") for k in range(2)]
    refs = [orc.moment(h, shape, dtype) for h in data]
    scales = [moment_scale(h, shape, dtype) for h in data]
    devs = [to_dev(h, dtype, shape) for h in data]
    # p, then different data of the same shape, then p again: a partial the kernel failed
    # to write would still hold the previous call's value and show up as a mismatch
    for k in (0, 1, 0, 1):
        out = torch.full((len(shape) + 1,), np.nan, dtype=torch.float64, device="cuda")
        got = _noalloc(tr, devs[k], out).cpu().numpy()
        check_moment(got, refs[k], scales[k], TOL[dtype])
        ws_result = tr.triot_moment(devs[k]).cpu().numpy()
        assert got.tobytes() == ws_result.tobytes()


@pytest.mark.parametrize("dtype,shape", [("f64", (9,) * 8), ("f32", (2,) * 24)])
def test_noalloc_default_plans_of_the_workloads_fit(tr, dtype, shape):
    """The default plans of the f64 d=8 and f32 d=24 moments fit the scratch."""
    n = int(np.prod(shape))
    ph = synth.normalise(synth.uniform01(9200, n))
    if dtype == "f32":
        ph = ph.astype(np.float32)
    p = torch.from_numpy(ph.reshape(shape)).cuda()
    out = torch.full((len(shape) + 1,), np.nan, dtype=torch.float64, device="cuda")
    got = _noalloc(tr, p, out).cpu().numpy()
    assert got.tobytes() == tr.triot_moment(p).cpu().numpy().tobytes()
    ref = orc.moment(ph, shape, dtype, nthreads=8)
    check_moment(got, ref, np.abs(ref), TOL[dtype])


def test_noalloc_empty_and_too_large(tr):
    out = torch.full((3,), np.nan, dtype=torch.float64, device="cuda")
    p = torch.empty((4, 0), dtype=torch.float32, device="cuda")
    assert np.all(_noalloc(tr, p, out).cpu().numpy() == 0.0)
    # rank 24 with many blocks and 32 CTAs per SM forced needs more partials than the
    # scratch holds: the call is refused and enqueues nothing
    L = tr.lib()
    shape = (2,) * 23 + (24,)
    q = torch.ones(shape, dtype=torch.float16, device="cuda")
    tr.triot_tune_set(tr.OP_MOMENT, shape, None, torch.float16, ctas_per_sm=32)
    try:
        out2 = torch.full((25,), np.nan, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        st = L.triot_moment_noalloc(24, tr._shape(shape), q.data_ptr(), 3, out2.data_ptr(), None)
        assert st == 5 and "scratch" in L.triot_last_error().decode()
        torch.cuda.synchronize()
        assert torch.isnan(out2).all()
    finally:
        tr.triot_tune_clear()
