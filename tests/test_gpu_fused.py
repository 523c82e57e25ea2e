"""Phases 3 and 4 fused (each S segment joined while its sort holds it in shared
memory) against the unfused kernels and the oracle."""
import numpy as np
import pytest

import gen
import oracle
from helpers import to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_0145_gb300 import Plan, mpsm as M  # noqa: E402


def cases():
    rng = np.random.default_rng(77)
    out = [gen.plain(70_000, 300_000, seed=1), gen.zipf(50_000, 400_000, 0.9, seed=2),
           gen.zipf(2_000, 300_000, 1.2, seed=3), gen.sparse(60_000, 90_000, seed=4),
           gen.plain(1, 5000, seed=5), gen.plain(300_000, 1, seed=6), gen.plain(9000, 9000, seed=7)]
    out = [(w.r_host(), w.s_host()) for w in out]
    # M:N with duplicates on both sides and the extreme keys
    for n_r, n_s, k in [(5000, 20000, 7), (40000, 40000, 300), (100, 100000, 3)]:
        R = np.zeros((n_r, 2), dtype=np.uint64)
        S = np.zeros((n_s, 2), dtype=np.uint64)
        keys = np.array([0, 1, 2**63, 2**64 - 2, 2**64 - 1] + list(rng.integers(0, 2**64 - 1, k, dtype=np.uint64)),
                        dtype=np.uint64)
        R[:, 0] = rng.choice(keys, n_r)
        S[:, 0] = rng.choice(keys, n_s)
        R[:, 1] = rng.integers(0, 2**64 - 1, n_r, dtype=np.uint64)
        S[:, 1] = rng.integers(0, 2**64 - 1, n_s, dtype=np.uint64)
        out.append((R, S))
    return out


@pytest.mark.parametrize("runs", [0, 1, 7, 300])
def test_fused_equals_unfused_and_oracle(runs):
    with Plan(1 << 19, 1 << 19, runs_r=runs) as f, Plan(1 << 19, 1 << 19, runs_r=runs, flags=M.FLAG_UNFUSED) as u:
        for R, S in cases():
            want = oracle.join(R, S)
            r, s = to_dev(R), to_dev(S)
            assert f.join(r, s) == want
            assert u.join(r, s) == want


def test_fused_batch_and_learned():
    ws = [gen.plain(3000 * (i + 1), 9000 * (i + 1), seed=40 + i) if i % 2 else
          gen.zipf(2000 * (i + 1), 16000 * (i + 1), 0.8, seed=40 + i) for i in range(9)]
    jobs = [(to_dev(w.r_host()), to_dev(w.s_host())) for w in ws]
    want = [oracle.join(w.r_host(), w.s_host()) for w in ws]
    tr = sum(w.n_r for w in ws)
    ts = sum(w.n_s for w in ws)
    for kw in ({}, {"flags": M.FLAG_UNFUSED}, {"splitter_mode": 1, "search_mode": 1}):
        with Plan(tr, ts, max_jobs=len(ws), **kw) as p:
            c, k = p.join_batch(jobs)
            assert list(zip(c, k)) == want, kw
            c, k = p.join_batch(jobs)
            assert list(zip(c, k)) == want, kw


def test_pairs_still_use_the_unfused_path():
    w = gen.zipf(10_000, 60_000, 0.9, seed=9)
    R, S = w.r_host(), w.s_host()
    with Plan(w.n_r, w.n_s) as p:
        cnt, chk = p.join(to_dev(R), to_dev(S))
        assert (cnt, chk) == oracle.join(R, S)


def test_fused_piece_of_equal_keys_inside_a_mixed_segment():
    """One partition of 6000 S tuples, the first 5000 with key 2: the fused kernel
    joins it in pieces of 4096, the first of which holds a single key while the
    segment's R windows also hold key 3."""
    R = np.array([[1, 11], [2, 22], [3, 33], [4, 44]], dtype=np.uint64)
    S = np.zeros((6000, 2), dtype=np.uint64)
    S[:5000, 0] = 2
    S[5000:, 0] = 3
    S[:, 1] = np.arange(6000, dtype=np.uint64) * 7919
    want = oracle.join(R, S)
    with Plan(16, 8192, partitions_s=1, runs_r=1) as p:
        assert p.join(to_dev(R), to_dev(S)) == want


@pytest.mark.parametrize("n_s", [8 << 20, 1 << 20, 500_000, 128_000, 8_000])
def test_fused_directory_widths(n_s):
    # R holds 2M dense unique keys, so a segment of about 3840 S tuples spans about
    # 3840 * 2M / |S| key values: 1K (the counting pass's exact directory), 8K and 15K
    # (one u16 directory entry per key), 60K and beyond (several keys per entry, a
    # bisection inside the entry)
    w = gen.plain(2 << 20, n_s, seed=97)
    R, S = w.r_host(), w.s_host()
    want = oracle.join(R, S)
    with Plan(w.n_r, w.n_s) as p:
        assert p.join(to_dev(R), to_dev(S)) == want
        assert p.device_errors() == 0


@pytest.mark.parametrize("theta", [0.8, 1.3])
def test_fused_wide_segments_with_hot_keys(theta):
    # few S tuples against many R keys and Zipf duplicates: wide directory entries hold
    # runs of equal keys
    w = gen.zipf(2 << 20, 300_000, theta, seed=98)
    R, S = w.r_host(), w.s_host()
    with Plan(w.n_r, w.n_s) as p:
        assert p.join(to_dev(R), to_dev(S)) == oracle.join(R, S)
        assert p.device_errors() == 0
