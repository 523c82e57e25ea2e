"""The learned first sort pass over the runs (MPSM_RUNS_LEARNED), element by element.

The pass cuts each run into buckets at the quantiles of a sorted run-side sample
instead of equal-width key ranges (Sec. 3.2.1 radix clustering with the empirical
CDF of Sec. 4.1-4.2).  The sorted runs must equal the oracle's, whatever the key
distribution, and clustered keys must need fewer passes than with equal-width
buckets.
"""
import numpy as np
import pytest

import gen
import oracle
from tests.helpers import from_dev_ptr, random_tuples, same_multiset, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_0145_gb300 import mpsm as M  # noqa: E402
from paper_1207_0145_gb300 import Plan  # noqa: E402


def sorted_runs(R, T, **opt):
    with Plan(len(R), 16, runs_r=T, **opt) as p:
        p.sort_runs(to_dev(R))
        v = p.view()
        got = from_dev_ptr(v.r_runs, len(R))
        off = from_dev_ptr(v.run_offsets, T + 1, width=1)
        return got, off, p.stats()["levels_r"]


def test_sparse_runs_take_fewer_passes_and_match_the_oracle():
    w = gen.sparse(1 << 21, 1 << 21, seed=81)
    R = w.r_host()
    want, want_off = oracle.sort_runs(R, 2)
    got0, off0, lv0 = sorted_runs(R, 2)
    got1, off1, lv1 = sorted_runs(R, 2, run_buckets=M.RUNS_LEARNED)
    assert (off1 == want_off).all() and (off0 == want_off).all()
    assert (got1 == want).all() and (got0 == want).all()  # unique keys: the sorted runs are unique
    assert lv0 >= 3 and lv1 <= 2 and lv1 < lv0, (lv0, lv1)


@pytest.mark.parametrize("T", [1, 3, 7])
def test_uniform_and_ragged_runs(T):
    w = gen.plain(700_001, 16, seed=82)
    R = w.r_host()
    want, want_off = oracle.sort_runs(R, T)
    got, off, lv = sorted_runs(R, T, run_buckets=M.RUNS_LEARNED)
    assert (off == want_off).all()
    assert (got == want).all()


@pytest.mark.parametrize("domain", [3, 40, 5000])
def test_hot_keys_equal_to_many_quantiles(domain):
    # few distinct keys: every key equals many quantiles and goes whole to the first
    # bucket they bound (a constant child); the runs must still come out sorted
    rng = np.random.default_rng(83 + domain)
    R = random_tuples(rng, 600_000, domain)
    R[:1000, 0] = np.uint64(2**64 - 1)  # the largest key, in the first run only
    T = 2
    want, off_want = oracle.sort_runs(R, T)
    got, off, _ = sorted_runs(R, T, run_buckets=M.RUNS_LEARNED)
    assert (off == off_want).all()
    assert (got[:, 0] == want[:, 0]).all()
    for j in range(T):
        a, b = int(off[j]), int(off[j + 1])
        assert same_multiset(got[a:b], want[a:b])


def test_keys_outside_the_sample_range():
    # the sample misses the extremes: a key below the smallest sampled key takes the
    # first bucket, one above the largest the last
    rng = np.random.default_rng(84)
    R = random_tuples(rng, 400_000, 1 << 40)
    R[1::64, 0] = np.uint64(0)          # rows the evenly spaced sample does not take
    R[3::64, 0] = np.uint64(2**64 - 1)
    want, want_off = oracle.sort_runs(R, 1)
    got, off, _ = sorted_runs(R, 1, run_buckets=M.RUNS_LEARNED)
    assert (got[:, 0] == want[:, 0]).all()
    assert same_multiset(got, want)


@pytest.mark.parametrize("w", [gen.sparse(1 << 20, 1 << 21, seed=85), gen.zipf(1 << 20, 1 << 22, 0.9, seed=86),
                               gen.plain(1 << 20, 1 << 22, seed=87)])
def test_joins_with_learned_runs(w):
    R, S = w.r_host(), w.s_host()
    want = oracle.join(R, S)
    for opt in ({}, {"splitter_mode": M.SPLIT_LEARNED, "search_mode": M.SEARCH_LEARNED},
                {"flags": M.FLAG_UNFUSED}):
        with Plan(w.n_r, w.n_s, runs_r=2, run_buckets=M.RUNS_LEARNED, **opt) as p:
            assert p.join(to_dev(R), to_dev(S)) == want, opt
            assert p.device_errors() == 0


def test_host_buffers_in_pieces_with_learned_runs():
    # 2^28 partitioned tuples take the piecewise host join (four pieces of 2^26)
    w = gen.sparse(1 << 24, 1 << 28, seed=88)
    R = torch.empty((w.n_r, 2), dtype=torch.int64, device="cuda")
    S = torch.empty((w.n_s, 2), dtype=torch.int64, device="cuda")
    w.fill_r_device(R.data_ptr(), torch.cuda.current_stream().cuda_stream)
    w.fill_s_device(S.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    Rh = torch.from_numpy(M.host_tuples(w.n_r).view(np.int64))
    Sh = torch.from_numpy(M.host_tuples(w.n_s).view(np.int64))
    Rh.copy_(R)
    Sh.copy_(S)
    del R, S
    with Plan(w.n_r, w.n_s, run_buckets=M.RUNS_LEARNED) as p:
        assert p.join_host(Rh, Sh) == oracle.closed_form(w)
        assert p.device_errors() == 0


def test_batch_jobs_each_take_their_own_bucket_function():
    jobs = [gen.sparse(300_000, 200_000, seed=89), gen.plain(500_000, 900_000, seed=90),
            gen.zipf(250_000, 600_000, 1.1, seed=91)]
    hosts = [(w.r_host(), w.s_host()) for w in jobs]
    nR = sum(len(r) for r, _ in hosts)
    nS = sum(len(s) for _, s in hosts)
    with Plan(nR, nS, max_jobs=len(jobs), runs_r=3, run_buckets=M.RUNS_LEARNED) as p:
        counts, sums = p.join_batch([(to_dev(r), to_dev(s)) for r, s in hosts])
    assert list(zip(counts, sums)) == [oracle.join(r, s) for r, s in hosts]


@pytest.mark.parametrize("w", [gen.plain(1 << 18, 1 << 21, seed=94), gen.zipf(1 << 18, 1 << 21, 1.1, seed=95)])
def test_reversed_roles_sort_the_foreign_keys_into_runs(w):
    # with R partitioned, S is cut into runs: its foreign keys repeat (hot keys under
    # Zipf), so the learned run buckets meet keys equal to many boundaries
    R, S = w.r_host(), w.s_host()
    with Plan(w.n_r, w.n_s, partition_side=M.PART_R, runs_r=3, run_buckets=M.RUNS_LEARNED) as p:
        assert p.join(to_dev(R), to_dev(S)) == oracle.join(R, S)
        assert p.device_errors() == 0


def test_short_runs_take_no_sort_pass():
    # runs of at most 8192 tuples are sorted in shared memory directly; the option is inert
    w = gen.plain(200_000, 800_000, seed=96)
    R, S = w.r_host(), w.s_host()
    with Plan(w.n_r, w.n_s, runs_r=64, run_buckets=M.RUNS_LEARNED) as p:
        assert p.join(to_dev(R), to_dev(S)) == oracle.join(R, S)
        assert p.stats()["levels_r"] == 0
