"""Failure detection without a GPU fault: a bounded device wait that runs out is reported
through triot_device_status, the flag clears on reading, and the context stays usable."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tr():
    from paper_1608_00099_gb300 import build, triot
    build.build()
    triot.lib()
    return triot


def test_wait_time_out_sets_and_clears_device_status(tr):
    assert tr.triot_device_status() == 0
    tr.triot_selftest_wait_timeout(8)
    assert tr.triot_device_status() == 9          # TRIOT_ERR_DEVICE
    assert "guard" in tr.lib().triot_last_error().decode()
    assert tr.triot_device_status() == 0          # reading cleared it
    # the context still works: a moment after the time-out is right
    p = torch.ones((3, 4), dtype=torch.float64, device="cuda")
    m = tr.triot_moment(p).cpu().numpy()
    assert np.array_equal(m, [12.0 * 1.0, 12.0 * 1.5, 12.0])
    assert tr.triot_device_status() == 0


def test_selftest_limit_checked_on_host(tr):
    import ctypes as C
    assert tr.lib().triot_selftest_wait_timeout(0, None) == 8
    assert tr.lib().triot_selftest_wait_timeout(5000, None) == 8
