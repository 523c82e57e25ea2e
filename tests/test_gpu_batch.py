"""Batched joins: the autotuner's candidates all give the per-job oracle result, the
chosen tuning stays on the plan, a replayed graph reports its kernel count, and a
learned-mode batch matches too."""
import numpy as np
import pytest

import gen
import oracle
from helpers import to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_0145_gb300 import Plan  # noqa: E402


def make_jobs(n, seed):
    rng = np.random.default_rng(seed)
    jobs, want = [], []
    for i in range(n):
        nr = int(np.exp(rng.uniform(np.log(2000), np.log(200_000))))
        w = gen.Workload(gen.KIND_ZIPF if i % 2 else gen.KIND_UNIFORM, nr, nr * int(rng.choice([1, 2, 4, 8, 16])),
                         seed=900 + i + seed, theta=0.8)
        R, S = w.r_host(), w.s_host()
        want.append(oracle.join(R, S))
        jobs.append((to_dev(R), to_dev(S)))
    return jobs, want


def test_autotuned_batch_matches_oracle():
    jobs, want = make_jobs(24, 1)
    tr = sum(len(r) for r, _ in jobs)
    ts = sum(len(s) for _, s in jobs)
    with Plan(tr, ts, max_jobs=len(jobs)) as p:
        best, ms = p.autotune(jobs, reps=1)
        assert best["radix_bits"] in (9, 11) and best["join_tile"] in (2048, 4096) and ms > 0
        c, k = p.join_batch(jobs)
        assert list(zip(c, k)) == want
        assert p.stats()["launches"] > 0
        c2, k2 = p.join_batch(jobs)  # replay of the tuned graph
        assert (c2, k2) == (c, k) and p.stats()["launches"] > 0
        # sequential single joins on the same plan agree
        p.set_tuning()
        assert [p.join(r, s) for r, s in jobs[:6]] == want[:6]


@pytest.mark.parametrize("opts", [{"search_mode": 2}, {"splitter_mode": 2}, {"splitter_mode": 2, "search_mode": 2}])
def test_batch_with_interpolation_search_and_equi_height_splitters(opts):
    jobs, want = make_jobs(12, 3)
    tr = sum(len(r) for r, _ in jobs)
    ts = sum(len(s) for _, s in jobs)
    with Plan(tr, ts, max_jobs=len(jobs), **opts) as p:
        for _ in range(2):  # capture, then replay
            c, k = p.join_batch(jobs)
            assert list(zip(c, k)) == want


def test_learned_batch_matches_oracle():
    jobs, want = make_jobs(10, 2)
    tr = sum(len(r) for r, _ in jobs)
    ts = sum(len(s) for _, s in jobs)
    with Plan(tr, ts, max_jobs=len(jobs), splitter_mode=1, search_mode=1) as p:
        c, k = p.join_batch(jobs)
        assert list(zip(c, k)) == want
        c, k = p.join_batch(jobs)
        assert list(zip(c, k)) == want
