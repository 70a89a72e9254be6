"""Failure detection on the GPU without a fault: the bounded wait of the streaming-strip
kernel on its bulk-copy barriers ends whether or not the barrier completes, and a wait
that ran out reaches the host as the timeout bit of the error word (LB_E_TIMEOUT from the
step calls).  The barrier that runs out is one that nothing ever completes.  The same for
the chained steps' wait on a neighbouring tile's completion flag: a flag that nothing
writes ends the wait after its bound with the stall bit."""
import time

import pytest

pytestmark = pytest.mark.gpu


def test_bounded_wait_completes_or_reports_timeout(gpu_lib):
    from paper_1805_07251_gb300 import capi

    assert capi.lb_selftest_wait(0, 1000, 1) == 0            # thread 0 arrives: completes
    t0 = time.perf_counter()
    assert capi.lb_selftest_wait(0, 1000, 0) == 2            # nobody arrives: the polls run out
    assert time.perf_counter() - t0 < 10.0
    with pytest.raises(capi.LBError):
        capi.lb_selftest_wait(0, 0, 0)                       # polls < 1 is refused


def test_bounded_flag_wait_completes_or_reports_stall(gpu_lib):
    from paper_1805_07251_gb300 import capi

    assert capi.lb_selftest_flag_wait(0, 1_000_000, 1) == 0          # the flag holds the step
    t0 = time.perf_counter()
    assert capi.lb_selftest_flag_wait(0, 2_000_000, 0) == 4          # never written: 2 ms, stall bit
    assert time.perf_counter() - t0 < 10.0
    for bad in (0, 10**11):
        with pytest.raises(capi.LBError):
            capi.lb_selftest_flag_wait(0, bad, 0)
