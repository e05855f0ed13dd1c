"""Naive multidimensional convolution (Alg 14/15, benchmark 4) against the oracle's scatter in
the paper's loop order, which is pinned against scipy.signal.convolve.  Tolerance: the sums
differ only in order, |got - want| <= 1e-13 * (|a| conv |b|)[t]."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1608_00099_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tr():
    from paper_1608_00099_gb300 import build, triot
    build.build()
    triot.lib()
    assert torch.cuda.is_available()
    return triot


CASES = [
    ((2 ** 8, 2 ** 3), (2 ** 8, 2 ** 3)),   # benchmark 4
    ((5,), (7,)),
    ((1,), (1,)),
    ((3, 4, 5), (2, 6, 3)),
    ((40, 1, 7), (3, 5, 9)),
    ((2, 3, 2, 3), (3, 2, 3, 2)),
    ((300,), (1000,)),
    ((0, 4), (3, 5)),                       # empty a on axis 0: result (2, 8) of zeros
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_convolve_matches_oracle(tr, case):
    sa, sb = CASES[case]
    a = synth.normal01(900 + case, int(np.prod(sa)))
    b = synth.normal01(950 + case, int(np.prod(sb)))
    got = tr.triot_convolve(torch.from_numpy(a.reshape(sa)).cuda(), torch.from_numpy(b.reshape(sb)).cuda())
    got = got.cpu().numpy().reshape(-1)
    if 0 in sa or 0 in sb:
        assert np.all(got == 0.0)
        return
    want = orc.convolve_f64(a, sa, b, sb).reshape(-1)
    scale = orc.convolve_f64(np.abs(a), sa, np.abs(b), sb).reshape(-1)
    assert np.all(np.abs(got - want) <= 1e-13 * scale + 1e-300)


def test_convolve_deterministic_and_exact_on_integers(tr):
    """Small integers: every product and partial sum is exact, so the result is exact."""
    rng = np.random.default_rng(5)
    sa, sb = (17, 6), (9, 11)
    a = rng.integers(-5, 6, size=int(np.prod(sa))).astype(np.float64)
    b = rng.integers(-5, 6, size=int(np.prod(sb))).astype(np.float64)
    A, B = torch.from_numpy(a.reshape(sa)).cuda(), torch.from_numpy(b.reshape(sb)).cuda()
    g1 = tr.triot_convolve(A, B).cpu().numpy()
    g2 = tr.triot_convolve(A, B).cpu().numpy()
    assert g1.tobytes() == g2.tobytes()
    assert g1.reshape(-1).tobytes() == orc.convolve_f64(a, sa, b, sb).reshape(-1).tobytes()
