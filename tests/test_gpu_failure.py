"""Failure detection on the GPU without a fault: a bounded device wait runs out.

The binning's wait on a row another CTA is writing gives up after a number of polls,
sets LS_ERR_TIMEOUT in the sticky status and lets the kernel return.  Here the wait
runs on a flag that nothing sets (ls_probe_wait) under a short limit, so it must run
out; the context stays usable, a flag that is already set passes, a binning call
under the short limit returns with a status that agrees with its own counters, and
after the default limit is restored the same binning is bit-exact again."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import assert_bins_equal, to_device

pytestmark = pytest.mark.gpu

LS_ERR_TIMEOUT = -4


@pytest.fixture(scope="module")
def lsb():
    import paper_2509_20198_b300 as lsb
    from paper_2509_20198_b300 import build
    build.build_library()
    return lsb


def test_bounded_wait_runs_out_and_the_context_stays_usable(lsb):
    import torch
    region = synth.Region(tiles_x=3, tiles_y=3)
    counts = synth.lognormal_counts(61, 9)
    pts = synth.region_points(61, region, counts)
    d = to_device(pts)
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    lsb.last_error()
    lsb.bin_stats(reset=True)
    try:
        lsb.set_spin_limit(1000)
        lsb.probe_wait(flag)                      # nothing ever sets the flag
        assert lsb.last_error() == LS_ERR_TIMEOUT
        st = lsb.bin_stats(reset=True)
        assert st["waits"] == 1 and st["wait_timeouts"] == 1
        assert lsb.last_error() == 0              # the status was read and cleared
        flag.fill_(2)
        lsb.probe_wait(flag)                      # already set: no wait at all
        assert lsb.last_error() == 0
        assert lsb.bin_stats(reset=True)["waits"] == 0
        # binning under a one-poll limit: every kernel returns; the status reports a
        # timeout exactly when the kernel's counters saw one
        lsb.set_spin_limit(1)
        lsb.bin_points(d, region, levels=(640, 64))
        torch.cuda.synchronize()
        err = lsb.last_error()
        st = lsb.bin_stats(reset=True)
        print("binning under a one-poll limit:", st, "status", err)
        assert err in (0, LS_ERR_TIMEOUT)
        assert (err == LS_ERR_TIMEOUT) == (st["wait_timeouts"] > 0)
    finally:
        lsb.set_spin_limit(0)
    out, dropped = lsb.bin_points(d, region, levels=(640, 64))
    torch.cuda.synchronize()
    assert lsb.last_error() == 0
    assert lsb.bin_stats(reset=True)["wait_timeouts"] == 0
    for b, cells in zip(out, (640, 64)):
        assert_bins_equal(b, oracle.bin_points(pts, region, cells), msg=f"cells={cells}")
    assert int(dropped.item()) == 0


def test_spin_limit_and_probe_reject_bad_arguments(lsb):
    import torch
    from paper_2509_20198_b300 import _native as N
    assert N.lib().ls_probe_wait(None, None) == -1
    t = torch.zeros(4, dtype=torch.int32, device="cuda")
    assert N.lib().ls_probe_wait(t.data_ptr() + 2, None) == -1   # not 4-byte aligned
    assert N.lib().ls_set_spin_limit(0) == 0
    torch.cuda.synchronize()
    assert lsb.last_error() == 0
