"""Properties of the input generator (host side): bijections, key structure, draws."""
import numpy as np
import pytest

import gen


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 17, 255, 256, 1000, 4097, 65537])
def test_feistel_permutation_is_a_bijection(n):
    L = gen.lib()
    img = [L.gen_permute(i, n, 42, 1) for i in range(n)]
    assert sorted(img) == list(range(n))
    assert [L.gen_permute_inv(y, n, 42, 1) for y in img] == list(range(n))


def test_plain_workload_structure():
    w = gen.plain(10_000, 40_000, seed=3)
    R, S = w.r_host(), w.s_host()
    assert sorted(R[:, 0].tolist()) == list(range(1, 10_001))
    rows = w.s_rows_host().astype(np.int64)
    assert (S[:, 0] == R[rows, 0]).all()
    # deterministic and thread-count independent
    assert (w.s_host(nthreads=1) == w.s_host(nthreads=3)).all()
    assert (gen.plain(10_000, 40_000, seed=4).r_host() != R).any()


def test_zipf_workload_skew():
    w = gen.zipf(100_000, 400_000, 0.9, seed=1)
    R, S = w.r_host(), w.s_host()
    assert np.isin(S[:, 0], R[:, 0]).all()
    _, c = np.unique(S[:, 0], return_counts=True)
    c = np.sort(c)[::-1]
    harmonic = sum(k ** -0.9 for k in range(1, 100_001))
    assert abs(c[0] / len(S) - 1 / harmonic) < 0.1 / harmonic  # hottest key ~ 1/H_{N,theta}
    # hot keys sit at random positions of the key order, not at the small keys
    hot = S[:, 0][np.argmax(np.bincount(S[:, 0].astype(np.int64)))]
    assert hot != 1


def test_zipf_table_is_a_cdf():
    thr, lo = gen.zipf_table(1_000_000, 0.8)
    assert (thr[1:] >= thr[:-1]).all()
    assert thr[-1] == np.uint64(gen.GEN_NONE)
    assert lo[0] == 0 and lo[-1] == 1_000_000 and (lo[1:] > lo[:-1]).all()


def test_sparse_workload_structure():
    w = gen.sparse(30_000, 50_000, fk_share=0.7, seed=12)
    R, S = w.r_host(), w.s_host()
    keys = np.sort(R[:, 0])
    assert len(np.unique(keys)) == len(keys)
    assert (np.diff(keys) >= 2).all()  # every gap holds a non-key
    spec = w.host_spec()
    L = gen.lib()
    sorted_keys = np.array([L.gen_sorted_key(spec, g) for g in range(len(keys))], dtype=np.uint64)
    assert (sorted_keys == keys).all()
    rows = w.s_rows_host()
    fk = rows != np.uint64(gen.GEN_NONE)
    assert fk.sum() == w.n_fk
    assert (S[fk, 0] == R[rows[fk].astype(np.int64), 0]).all()
    assert not np.isin(S[~fk, 0], R[:, 0]).any()
    # spread over the whole 64-bit domain: top bits vary
    assert len(np.unique(keys >> np.uint64(58))) >= 32


def test_negcorr_workload_skew():
    # Sec. 5.6: 80 % of R's keys in the low fifth of the domain, 80 % of S's in the high fifth
    w = gen.negcorr(100_000, 400_000, seed=5)
    R, S = w.r_host(), w.s_host()
    keys = np.sort(R[:, 0])
    lo = 4 * 100_000 // 5
    assert keys[:lo].tolist() == list(range(1, lo + 1))
    assert (np.diff(keys[lo:]) == 16).all()
    top = int(keys[-1])
    assert abs(np.mean(R[:, 0] <= top // 5) - 0.8) < 1e-3
    assert abs(np.mean(S[:, 0] > top * 4 // 5) - 0.8) < 0.01
    rows = w.s_rows_host().astype(np.int64)
    assert (S[:, 0] == R[rows, 0]).all()  # foreign keys
    # R's keys in random order (not sorted by row)
    assert (np.diff(R[:, 0].astype(np.int64)) < 0).any()
    for n in (1, 2, 3, 7):
        t = gen.negcorr(n, 50, seed=9)
        r, s2 = t.r_host(), t.s_host()
        assert np.isin(s2[:, 0], r[:, 0]).all()


def test_locskew_workload_structure():
    # Sec. 5.5: small to large key order by clusters, no order inside a cluster
    n = 100_003
    w = gen.locskew(n, 300_000, seed=6)
    R, S = w.r_host(), w.s_host()
    assert sorted(R[:, 0].tolist()) == list(range(1, n + 1))
    for c in range(64):
        a, b = n * c // 64, n * (c + 1) // 64
        blk = R[a:b, 0]
        assert sorted(blk.tolist()) == list(range(a + 1, b + 1))
        assert (np.diff(blk.astype(np.int64)) < 0).any()
    rows = w.s_rows_host().astype(np.int64)
    assert (S[:, 0] == R[rows, 0]).all()
    for m in (1, 2, 63, 64, 65, 130):
        t = gen.locskew(m, 40, seed=2)
        assert sorted(t.r_host()[:, 0].tolist()) == list(range(1, m + 1))


def test_batch_jobs_shape():
    jobs = gen.batch_jobs(256)
    nr = np.array([j.n_r for j in jobs])
    assert nr.min() >= 10 * 1024 and nr.max() <= 20 * gen.M
    mult = {j.n_s // j.n_r for j in jobs}
    assert mult <= {1, 2, 4, 8, 16}
    assert sum(j.kind == gen.KIND_ZIPF for j in jobs) == 128
