"""Failure paths on the GPU, exercised without faulting or hanging it: a bounded device wait
that runs out (the kernel sets its status word and returns), allocation failures and refused
arguments reported as error codes, and the device still usable afterwards."""
import numpy as np
import pytest

import oracle
from paper_0901_1307_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SECTOR = 512


@pytest.fixture(scope="module")
def cv(cuda_device):
    import __graft_entry__

    __graft_entry__.build()
    from paper_0901_1307_gb300 import cv as cvmod

    return cvmod


def test_bounded_wait_times_out_and_device_stays_usable(cv):
    assert cv.selftest_wait_timeout(20000) == cv.CV_ETIMEOUT
    assert cv.selftest_wait_timeout(0) == cv.CV_EINVAL
    plan = synth.config_plan("small:3000:10:61")
    files = plan.masters_host()
    img = plan.image_host()
    with cv.master_build(files) as m, cv.scan(m, [torch.from_numpy(img).cuda()]) as r:
        assert np.array_equal(r.matches(0), oracle.match_hash(img, files))


def test_allocation_failures_are_error_codes(cv):
    files = [synth.random_sectors(7, 32)]
    with cv.master_build(files) as m:
        with pytest.raises(cv.CVError) as e:
            cv.server_create(m, hbm_budget_bytes=1 << 50, work_unit_bytes=1 << 30)
        assert e.value.code in (cv.CV_ENOMEM, cv.CV_EINVAL)
        with pytest.raises(cv.CVError) as e:
            cv.batch_create(m, [np.ascontiguousarray(files[0])])  # host image: batches are device-only
        assert e.value.code == cv.CV_EINVAL
        with cv.scan(m, [torch.from_numpy(files[0]).cuda()]) as r:
            assert r.count(0) == 32


def test_int_peak_measures_both_pipes(cv):
    p = cv.int_peak()
    assert p["sms"] > 0 and p["sm_clock_mhz"] > 500
    per_clk = lambda x: x / (p["sms"] * p["sm_clock_mhz"] * 1e6)
    # one operation per lane per two clocks on each pipe; interleaving both approaches four
    # schedulers x 32 lanes
    assert 40 < per_clk(p["alu_ops_per_s"]) < 70
    assert per_clk(p["mixed_ops_per_s"]) > per_clk(p["alu_ops_per_s"])
