"""The allocation-free run sort (mpsm_sort_runs_noalloc) against mpsm_sort_runs and the oracle.

Some callers cannot allocate device memory (a framework owns the pool, or a
cudaMalloc's device-wide synchronisation is not acceptable on their path); for
them the library sorts a small R's runs with scratch kept in a fixed device
array.  This file runs last so that a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest

import gen
import oracle
from tests.helpers import from_dev_ptr, random_tuples, same_multiset, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_0145_gb300 import Plan  # noqa: E402
from paper_1207_0145_gb300 import mpsm as M  # noqa: E402


def reference_runs(R_host, runs):
    with Plan(len(R_host), 1, runs_r=runs) as p:
        p.sort_runs(to_dev(R_host))
        v = p.view()
        return from_dev_ptr(v.r_runs, len(R_host)), from_dev_ptr(v.run_offsets, runs + 1, width=1)


def test_noalloc_sort_matches_plan_sort_twice():
    w = gen.plain(200_000, 10, seed=77)  # unique keys: the sorted runs are unique
    R_host = w.r_host()
    runs = 40  # 5000 tuples per run
    want, off = reference_runs(R_host, runs)
    R = to_dev(R_host)
    for call in range(2):  # the shared scratch keeps the last call's contents
        out = torch.full_like(R, -1)
        M.sort_runs_noalloc(R, runs, out)
        got = out.cpu().numpy().view(np.uint64)
        assert (got == want).all(), call


def test_noalloc_sort_duplicates_and_large_runs():
    rng = np.random.default_rng(5)
    R_host = random_tuples(rng, 3 * 8192 + 17, 300)  # runs just above 4096 and up to 8192, equal keys
    runs = 4
    want, off = reference_runs(R_host, runs)
    R = to_dev(R_host)
    for call in range(2):
        out = torch.zeros_like(R)
        M.sort_runs_noalloc(R, runs, out)
        got = out.cpu().numpy().view(np.uint64)
        assert (got[:, 0] == want[:, 0]).all(), call
        for j in range(runs):
            a, b = int(off[j]), int(off[j + 1])
            assert same_multiset(got[a:b], want[a:b])


def test_noalloc_sort_rejects_sizes_beyond_the_limit():
    R = torch.zeros((2 * 8192 + 1, 2), dtype=torch.int64, device="cuda")
    out = torch.zeros_like(R)
    with pytest.raises(M.MPSMError) as e:
        M.sort_runs_noalloc(R, 2, out)  # a run of 8193 tuples
    assert e.value.status == M.ERR_INVALID_ARG
    with pytest.raises(M.MPSMError):
        M.sort_runs_noalloc(R, 1025, out)
    rc = M.lib().mpsm_sort_runs_noalloc(R.data_ptr() + 8, 10, 1, out.data_ptr(), None)
    assert rc == M.ERR_INVALID_ARG  # misaligned


@pytest.mark.parametrize("run_len", [4096, 8192])
def test_noalloc_sort_in_place_matches_oracle(run_len):
    # out == R (allowed by the header), runs of exactly 4096 and 8192 tuples, equal keys
    rng = np.random.default_rng(run_len)
    runs = 5
    R_host = random_tuples(rng, runs * run_len, 1000)
    want, off = oracle.sort_runs(R_host, runs)
    R = to_dev(R_host)
    for call in range(2):
        M.sort_runs_noalloc(R, runs, R)
        got = R.cpu().numpy().view(np.uint64)
        assert (got[:, 0] == want[:, 0]).all(), call
        for j in range(runs):
            a, b = int(off[j]), int(off[j + 1])
            assert same_multiset(got[a:b], want[a:b]), (call, j)
        R = to_dev(R_host)


def test_noalloc_sort_matches_oracle_unique_keys():
    w = gen.plain(150_000, 10, seed=78)
    R_host = w.r_host()
    want, _ = oracle.sort_runs(R_host, 37)
    R = to_dev(R_host)
    out = torch.full_like(R, -1)
    M.sort_runs_noalloc(R, 37, out)
    assert (out.cpu().numpy().view(np.uint64) == want).all()
