"""Failure detection without a GPU fault: the bounded waits of the kernels give up
and report, and the context stays usable; a device-side check failure is reported
as MPSM_ERR_DEVICE with its MPSM_DEVERR_* bits."""
import numpy as np
import pytest

import gen
import oracle
from helpers import to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_0145_gb300 import Plan, mpsm as M  # noqa: E402


@pytest.mark.parametrize("limit", [1, 1000, 100_000])
def test_bounded_wait_gives_up_and_the_context_stays_usable(limit):
    rc, flags = M.selftest_wait_timeout(limit)
    assert rc == M.ERR_DEVICE and flags == M.DEVERR_WAIT_TIMEOUT
    w = gen.plain(20_000, 80_000, seed=41)
    R, S = w.r_host(), w.s_host()
    with Plan(w.n_r, w.n_s) as p:
        assert p.join(to_dev(R), to_dev(S)) == oracle.join(R, S)
        assert p.device_errors() == 0


def test_device_errors_are_cleared_by_a_good_call():
    w = gen.zipf(30_000, 90_000, 0.9, seed=42)
    R, S = w.r_host(), w.s_host()
    with Plan(w.n_r, w.n_s) as p:
        for _ in range(2):
            assert p.join(to_dev(R), to_dev(S)) == oracle.join(R, S)
            assert p.device_errors() == 0


@pytest.mark.parametrize("flags", [0, M.FLAG_UNFUSED])
def test_inexact_segment_bounds_are_reported_not_used(flags):
    # one final S segment's recorded key range narrowed on purpose: the sort kernels
    # check every key against it, report MPSM_DEVERR_BOUNDS and leave the segment
    # (every shared-memory index stays masked or range-checked; nothing faults)
    w = gen.plain(100_000, 400_000, seed=43)
    R, S = w.r_host(), w.s_host()
    want = oracle.join(R, S)
    with Plan(w.n_r, w.n_s, flags=flags | M.FLAG_BOUNDS_TEST) as p:
        with pytest.raises(M.MPSMError) as e:
            p.join(to_dev(R), to_dev(S))
        assert e.value.status == M.ERR_DEVICE
        assert p.device_errors() & M.DEVERR_BOUNDS
    with Plan(w.n_r, w.n_s, flags=flags) as p:  # the context stays usable
        assert p.join(to_dev(R), to_dev(S)) == want
        assert p.device_errors() == 0
