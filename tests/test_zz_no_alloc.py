"""The allocation-free moment entry point (triot_moment_noalloc).

Some callers cannot allocate device memory, so they cannot hand triot_moment a
workspace; triot_moment_noalloc keeps its partial sums in a fixed scratch array inside
the library instead.  This test calls it through the C ABI and checks it against
triot_moment (the workspace version) within the tolerances the other moment tests use,
on two calls in a row (the scratch keeps the previous call's contents).  It lives in a
file of its own that pytest collects last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5, torch.bfloat16: 1e-5}


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


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
def test_noalloc_matches_workspace_moment_twice(tr, dtype):
    g = torch.Generator(device="cpu").manual_seed(7)
    shapes = [(9, 9, 9, 9, 9), (37, 1, 41)]
    for shape in shapes:
        p = torch.rand(shape, generator=g, dtype=torch.float64).to(dtype).cuda()
        ref = tr.triot_moment(p).cpu().numpy()
        scale = np.abs(tr.triot_moment(p.abs()).cpu().numpy())
        for _ in range(2):   # two calls in a row share the scratch
            out = torch.full((p.dim() + 1,), np.nan, dtype=torch.float64, device="cuda")
            got = _noalloc(tr, p, out).cpu().numpy()
            assert np.all(np.abs(got - ref) <= TOL[dtype] * scale + 1e-300), (got, ref)


def test_noalloc_empty_and_too_large(tr):
    out = torch.full((3,), np.nan, dtype=torch.float64, device="cuda")
    p = torch.empty((4, 0), dtype=torch.float32, device="cuda")
    assert np.all(_noalloc(tr, p, out).cpu().numpy() == 0.0)
    # rank 24 with many blocks needs more partials than the scratch holds: with 32 CTAs per
    # SM allowed, 2^23 * 24 f16 elements take ~2700 CTAs * 25 partials > 65536
    L = tr.lib()
    shape = (2,) * 23 + (24,)
    q = torch.ones(shape, dtype=torch.float16, device="cuda")
    tr.triot_tune_set(tr.OP_MOMENT, shape, None, torch.float16, ctas_per_sm=32)
    try:
        out2 = torch.zeros(25, dtype=torch.float64, device="cuda")
        st = L.triot_moment_noalloc(24, tr._shape(shape), q.data_ptr(), 3, out2.data_ptr(), None)
        assert st == 5 and "scratch" in L.triot_last_error().decode()
    finally:
        tr.triot_tune_clear()
