"""Pins of the CPU oracle against facts that do not come from the oracle itself.

- the O(|R||S|) nested loop on tiny inputs (M:N duplicates, extreme keys, empty sides);
- closed forms of the generator's foreign-key workloads (count = |S| or the
  number of drawn tuples, checksum from the R row each S tuple was drawn from);
- the worked examples of Fig. 6 and Fig. 10 (histograms, prefix sums, splitters,
  scatter layout);
- exhaustive DP for the splitter objective, and numpy's searchsorted / stable
  argsort for the window and run oracles.
"""
import decimal
import math
import os

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U64 = (1 << 64) - 1


def golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, *v = line.split()
            vals[k] = [int(x) for x in v]
    return vals


def tuples(keys, payloads=None, seed=0):
    keys = np.asarray(keys, dtype=np.uint64)
    if payloads is None:
        payloads = np.random.default_rng(seed).integers(0, U64, len(keys), dtype=np.uint64, endpoint=True)
    return np.stack([keys, np.asarray(payloads, dtype=np.uint64)], axis=1)


def py_join(R, S):
    """Pair enumeration in pure Python integers (independent of both C++ loops)."""
    cnt, chk = 0, 0
    for rk, rp in R.tolist():
        for sk, sp in S.tolist():
            if rk == sk:
                cnt += 1
                chk = (chk + rp + sp) % (1 << 64)
    return cnt, chk


# ------------------------------------------------------------------ join vs brute force


def random_case(rng, nr, ns, domain):
    pool = np.array([0, U64, U64 - 1, 1, 1 << 63], dtype=np.uint64)
    kr = rng.integers(0, domain, nr, dtype=np.uint64)
    ks = rng.integers(0, domain, ns, dtype=np.uint64)
    if nr and rng.random() < 0.3:
        kr[rng.integers(0, nr, max(1, nr // 7))] = rng.choice(pool)
    if ns and rng.random() < 0.3:
        ks[rng.integers(0, ns, max(1, ns // 7))] = rng.choice(pool)
    R = tuples(kr, rng.integers(0, U64, nr, dtype=np.uint64, endpoint=True))
    S = tuples(ks, rng.integers(0, U64, ns, dtype=np.uint64, endpoint=True))
    return R, S


def test_join_matches_brute_force_random():
    rng = np.random.default_rng(7)
    for case in range(300):
        nr = int(rng.integers(0, 200))
        ns = int(rng.integers(0, 300))
        domain = int(rng.choice([1, 2, 5, 50, 1000, 1 << 40]))
        R, S = random_case(rng, nr, ns, domain)
        assert oracle.join(R, S) == oracle.brute(R, S), case


def test_join_matches_python_enumeration():
    rng = np.random.default_rng(11)
    for _ in range(40):
        R, S = random_case(rng, int(rng.integers(0, 40)), int(rng.integers(0, 40)), 6)
        assert oracle.join(R, S) == py_join(R, S)
        assert oracle.brute(R, S) == py_join(R, S)


def test_join_pairs_are_the_cross_products():
    rng = np.random.default_rng(3)
    R, S = random_case(rng, 60, 90, 9)
    c, k, pairs = oracle.join(R, S, with_pairs=True)
    want = sorted((int(rp), int(sp)) for rk, rp in R.tolist() for sk, sp in S.tolist() if rk == sk)
    assert c == len(want) == len(pairs)
    assert [tuple(map(int, p)) for p in pairs.tolist()] == want
    assert k == sum(a + b for a, b in want) % (1 << 64)


def test_join_edge_cases():
    e = np.zeros((0, 2), dtype=np.uint64)
    R = tuples([5, 5, 7])
    assert oracle.join(e, e) == (0, 0)
    assert oracle.join(R, e) == (0, 0) and oracle.join(e, R) == (0, 0)
    # all keys equal on both sides: |R| * |S| pairs
    R = tuples([9] * 13, range(13))
    S = tuples([9] * 17, range(100, 117))
    c, k = oracle.join(R, S)
    assert c == 13 * 17
    assert k == 17 * sum(range(13)) + 13 * sum(range(100, 117))
    # disjoint key ranges: no pairs
    assert oracle.join(tuples(range(10)), tuples(range(10, 20))) == (0, 0)
    # extreme keys, wrapping checksum
    R = tuples([0, U64], [U64, U64])
    S = tuples([U64, 0, 0], [2, 3, U64])
    assert oracle.join(R, S) == oracle.brute(R, S) == (3, (U64 + 2 + U64 + 3 + U64 + U64) % (1 << 64))


# ------------------------------------------------------------------ closed forms


def test_closed_form_plain_config0():
    """Config 'plain-1M-4M': R = permutation of 1..2^20, S = 4*2^20 uniform foreign keys.
    Every S tuple matches exactly one R tuple: count = |S| = 4,194,304."""
    w = gen.CONFIGS["plain-1M-4M"]()
    R, S = w.r_host(), w.s_host()
    c, k = oracle.join(R, S)
    assert c == 4 * (1 << 20) == 4194304
    # checksum from the generator's bookkeeping, summed in numpy (independent of oracle.cpp)
    rows = w.s_rows_host().astype(np.int64)
    want = (int(S[:, 1].sum(dtype=np.uint64)) + int(R[rows, 1].sum(dtype=np.uint64))) % (1 << 64)
    assert k == want
    assert oracle.closed_form(w) == (c, k)


@pytest.mark.parametrize("w", [gen.zipf(50_000, 200_000, 0.9, seed=5), gen.sparse(40_000, 60_000, seed=6),
                               gen.plain(3, 1000, seed=1), gen.zipf(1, 50, 0.8, seed=2),
                               gen.negcorr(60_000, 240_000, seed=7), gen.negcorr(2, 30, seed=8),
                               gen.locskew(50_003, 150_000, seed=9), gen.locskew(5, 40, seed=10)])
def test_closed_form_matches_join(w):
    R, S = w.r_host(), w.s_host()
    assert oracle.join(R, S) == oracle.closed_form(w)


def test_closed_form_sparse_count_is_fk_share():
    w = gen.sparse(20_000, 30_000, fk_share=0.7, seed=9)
    c, _ = oracle.closed_form(w)
    assert c == round(0.7 * 30_000) == w.n_fk


# ------------------------------------------------------------------ phase 1: runs


def test_sort_runs_matches_numpy_stable_sort():
    rng = np.random.default_rng(4)
    R = tuples(rng.integers(0, 50, 1000, dtype=np.uint64), np.arange(1000, dtype=np.uint64))
    for T in (1, 3, 7, 32):
        out, off = oracle.sort_runs(R, T)
        assert off[0] == 0 and off[-1] == len(R)
        for j in range(T):
            a, b = int(off[j]), int(off[j + 1])
            assert a == (len(R) * j) // T
            chunk = R[a:b]
            order = np.argsort(chunk[:, 0], kind="stable")
            assert (out[a:b] == chunk[order]).all()


# ------------------------------------------------------------------ phase 2: worked examples


def _chunked(g):
    keys = g["chunk1"] + g["chunk2"]
    S = tuples(keys, range(len(keys)))
    off = np.array([0, len(g["chunk1"]), len(keys)], dtype=np.uint64)
    return S, off


def test_fig6_histograms_and_prefix_sums():
    g = golden("fig6_partition.txt")
    nb, shift = oracle.fine_geometry(g["kmin"][0], g["kmax"][0], g["B"][0])
    assert nb == 2 and shift == 4  # the highest of 5 key bits
    S, off = _chunked(g)
    h = oracle.worker_histograms(S, off, g["kmin"][0], g["kmax"][0], shift, nb)
    assert h[0].tolist() == g["h1"]
    ps, part_off = oracle.prefix_sums(h)  # B = log T: one bucket per partition
    assert (ps[0] - part_off[:-1]).tolist() == g["ps1"]
    assert (ps[1] - part_off[:-1]).tolist() == g["ps2"]


def test_fig10_splitters_prefix_sums_and_scatter():
    g = golden("fig10_splitters.txt")
    kmin, kmax = g["kmin"][0], g["kmax"][0]
    nb, shift = oracle.fine_geometry(kmin, kmax, g["B"][0])
    assert nb == 4 and shift == 3  # buckets <8, [8,16), [16,24), >=24
    S, off = _chunked(g)
    h = oracle.worker_histograms(S, off, kmin, kmax, shift, nb)
    assert h[0].tolist() == g["h1"] and h[1].tolist() == g["h2"]
    H = h.sum(axis=0)
    assert H.tolist() == [7, 3, 3, 1]
    sp, nparts, best = oracle.splitters(H, np.array(g["other"], dtype=np.uint64), g["P"][0], g["T"][0])
    assert sp.tolist() == g["sp"] and nparts == 2
    # per-worker partition histograms, prefix sums, scatter
    hp = np.zeros((2, nparts), dtype=np.uint64)
    for f in range(nb):
        hp[:, sp[f]] += h[:, f]
    ps, part_off = oracle.prefix_sums(hp)
    assert np.diff(part_off).tolist() == g["parts"]
    assert (ps[0] - part_off[:-1]).tolist() == g["ps1"]
    assert (ps[1] - part_off[:-1]).tolist() == g["ps2"]
    out = oracle.scatter(S, off, kmin, kmax, shift, sp, ps)
    # partition 1 holds exactly the keys < 8, worker 1's first (in input order), then worker 2's
    assert out[:7, 0].tolist() == [0, 2, 5, 7, 1, 3, 6]
    assert out[7:, 0].tolist() == [12, 18, 21, 9, 14, 16, 27]


def test_fine_geometry_closed_form():
    # bucket = (key - kmin) >> shift with shift = max(0, bitlen(kmax - kmin) - B): the top B bits
    rng = np.random.default_rng(44)
    for _ in range(500):
        kmin = int(rng.integers(0, U64, dtype=np.uint64, endpoint=True))
        kmax = kmin + int(rng.integers(0, U64 - kmin + 1, dtype=np.uint64)) if kmin < U64 else U64
        B = int(rng.integers(1, 13))
        nb, shift = oracle.fine_geometry(kmin, kmax, B)
        assert shift == max(0, (kmax - kmin).bit_length() - B)
        assert nb == ((kmax - kmin) >> shift) + 1 and nb <= (1 << B)


def test_run_counts_against_searchsorted_and_brute_force():
    # the run side's tuples per fine bucket: its CDF at the bucket bounds (Sec. 4.1, 4.3),
    # read here by searchsorted in every sorted run and, on small inputs, by a plain loop
    rng = np.random.default_rng(45)
    for case in range(60):
        n = int(rng.integers(0, 4000))
        T = int(rng.integers(1, 10))
        domain = int(rng.choice([3, 100, 5000, 1 << 40, 1 << 64]))
        keys = (rng.integers(0, U64, n, dtype=np.uint64, endpoint=True) if domain == 1 << 64
                else rng.integers(0, domain, n, dtype=np.uint64))
        if n and case % 3 == 0:
            keys[rng.integers(0, n, max(1, n // 20))] = rng.choice(np.array([0, U64, U64 - 1], dtype=np.uint64))
        off = np.array([(n * j) // T for j in range(T + 1)], dtype=np.uint64)
        Rs = np.zeros((n, 2), dtype=np.uint64)
        for j in range(T):
            a, b = int(off[j]), int(off[j + 1])
            Rs[a:b, 0] = np.sort(keys[a:b])
        if n == 0:
            kmin, kmax = 5, 9
        elif case % 2:
            kmin, kmax = int(keys.min()), int(keys.max())
        else:  # a narrower range: keys outside it are not counted
            lo_, hi_ = sorted(int(x) for x in rng.choice(keys, 2))
            kmin, kmax = lo_, hi_
        B = int(rng.integers(1, 13))
        nb, shift = oracle.fine_geometry(kmin, kmax, B)
        G = oracle.run_counts(Rs, off, kmin, kmax, shift, nb)
        want = np.zeros(nb, dtype=np.int64)
        for j in range(T):
            run = Rs[int(off[j]):int(off[j + 1]), 0]
            # rank of each bound in the run; the last bucket ends after kmax
            lo = [int(np.searchsorted(run, np.uint64(kmin + (f << shift)), side="left")) for f in range(nb)]
            lo.append(int(np.searchsorted(run, np.uint64(kmax), side="right")))
            want += np.diff(np.array(lo, dtype=np.int64))
        assert (G.astype(np.int64) == want).all(), case
        if n <= 600:
            brute = [0] * nb
            for k in Rs[:, 0].tolist():
                if kmin <= k <= kmax:
                    brute[(k - kmin) >> shift] += 1
            assert G.tolist() == brute, case


# ------------------------------------------------------------------ phase 2: cost and solver


def exact_log2_q16(n: int) -> int:
    """floor(2^16 log2 n) from an 80-digit natural logarithm (Python's decimal rounds
    ln correctly); the fraction is asserted far from an integer, so the floor is certain."""
    if n <= 1:
        return 0
    if n & (n - 1) == 0:
        return (n.bit_length() - 1) << 16
    with decimal.localcontext() as ctx:
        ctx.prec = 80
        v = decimal.Decimal(n).ln() / decimal.Decimal(2).ln() * 65536
        f = int(v)
        frac = v - f
        assert decimal.Decimal("1e-60") < frac < 1 - decimal.Decimal("1e-60"), n
    return f


def boundary_n(L: int) -> int:
    """The smallest integer n with 2^16 log2 n >= L: where the floor steps to L."""
    with decimal.localcontext() as ctx:
        ctx.prec = 80
        return int((decimal.Decimal(2) ** (decimal.Decimal(L) / 65536)).to_integral_value(decimal.ROUND_CEILING))


def test_log2_q16_is_the_exact_floor():
    # the Q16 logarithm of the splitter cost is floor(2^16 log2 n), exactly (Sec. 4.3's n log n)
    rng = np.random.default_rng(41)
    ns = list(range(0, 1 << 13)) + [2 ** k + d for k in range(1, 64) for d in (-1, 0, 1)]
    ns += [int(x) for x in rng.integers(2, U64, 3000, dtype=np.uint64, endpoint=True)]
    ns += [int(x) >> int(s) for x, s in zip(rng.integers(2, U64, 2000, dtype=np.uint64), rng.integers(0, 62, 2000))]
    for n in ns:
        assert oracle.log2_q16(n) == exact_log2_q16(n), n


def test_log2_q16_at_the_steps_of_the_floor():
    # the n where floor(2^16 log2 n) changes: the hardest inputs for a finite-precision method
    rng = np.random.default_rng(42)
    for L in [int(x) for x in rng.integers(65536, 64 * 65536, 3000)] + [65536 * k + 1 for k in range(1, 64)]:
        n = boundary_n(L)
        if n > U64:
            continue
        # n is the first integer at or past the step to L (small n pass several steps at once)
        assert oracle.log2_q16(n) == exact_log2_q16(n) >= L, (L, n)
        assert oracle.log2_q16(n - 1) == exact_log2_q16(n - 1) < L, (L, n)
        if n > 1 << 17:  # consecutive integers there differ by less than one step
            assert oracle.log2_q16(n) == L, (L, n)


def test_log2_q16_invariants():
    rng = np.random.default_rng(43)
    for n in [int(x) for x in rng.integers(2, 1 << 32, 2000)]:
        a, b = oracle.log2_q16(n), oracle.log2_q16(n * n)
        assert b in (2 * a, 2 * a + 1), n  # floor(2x) is 2 floor(x) or one more
        assert oracle.log2_q16(2 * n) == a + 65536, n  # doubling adds exactly one
        assert oracle.log2_q16(n + 1) >= a
    for k in range(64):
        assert oracle.log2_q16(1 << k) == k << 16


def test_log2_q16_big_integer_definition():
    # the definition the interval method falls back to: bitlen(n^65536) - 1
    for n in (2, 3, 5, 7, 10, 100, 255, 1000, 4097):
        assert oracle.log2_q16_big(n) == exact_log2_q16(n) == oracle.log2_q16(n), n


def test_splitters_optimal_against_exhaustive_dp():
    rng = np.random.default_rng(21)
    for _ in range(300):
        nb = int(rng.integers(1, 11))
        P = int(rng.integers(1, 5))
        T = int(rng.integers(1, 40))
        H = rng.integers(0, 2000, nb, dtype=np.uint64)
        if rng.random() < 0.3:
            H[rng.integers(0, nb)] = rng.integers(10_000, 100_000)  # a hot bucket
        G = rng.integers(0, 500, nb, dtype=np.uint64)
        sp, nparts, best = oracle.splitters(H, G, P, T)
        assert best == oracle.splitters_dp(H, G, P, T)
        assert 1 <= nparts <= P
        assert sp[0] == 0 and (np.diff(sp.astype(np.int64)) >= 0).all() and (np.diff(sp.astype(np.int64)) <= 1).all()
        assert int(sp[-1]) == nparts - 1


def test_equi_height_splitters_against_exhaustive_dp_and_closed_forms():
    # kind 1 groups the buckets by the partitioned side's count alone (Sec. 5.6)
    rng = np.random.default_rng(22)
    for _ in range(300):
        nb = int(rng.integers(1, 11))
        P = int(rng.integers(1, 5))
        H = rng.integers(0, 2000, nb, dtype=np.uint64)
        G = rng.integers(0, 500, nb, dtype=np.uint64)
        sp, nparts, best = oracle.splitters(H, G, P, 7, kind=1)
        assert best == oracle.splitters_dp(H, G, P, 7, kind=1)
        sizes = np.bincount(sp, weights=H.astype(np.float64), minlength=nparts)
        assert int(sizes.max()) << 16 == best
        # the run side does not change the grouping
        assert (oracle.splitters(H, G[::-1].copy(), P, 7, kind=1)[0] == sp).all()
    # equal buckets split evenly: 12 buckets of 5 into 4 partitions of 3 buckets (15 tuples)
    sp, nparts, best = oracle.splitters(np.full(12, 5, dtype=np.uint64), np.zeros(12, dtype=np.uint64), 4, 3, kind=1)
    assert sp.tolist() == [0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3] and best == 15 << 16
    # ten unit buckets into three partitions: the largest holds ceil(10 / 3) = 4, leftmost greedy 4 + 4 + 2
    sp, nparts, best = oracle.splitters(np.ones(10, dtype=np.uint64), np.zeros(10, dtype=np.uint64), 3, 1, kind=1)
    assert best == 4 << 16 and sp.tolist() == [0, 0, 0, 0, 1, 1, 1, 1, 2, 2]


def test_equi_cost_differs_from_equi_height_under_negative_correlation():
    # Fig. 16a: the partitioned side dense at the high end, the run side dense at
    # the low end.  Equi-height gives the low partitions the wide key ranges (and so
    # most of the run side); equi-cost weighs the run side in, so its largest cost
    # is lower.
    nb, P, T = 64, 8, 32
    H = np.array([1] * 48 + [16] * 16, dtype=np.uint64) * 1000
    G = np.array([16] * 16 + [1] * 48, dtype=np.uint64) * 1000
    sp_h, _, _ = oracle.splitters(H, G, P, T, kind=1)
    sp_c, _, best_c = oracle.splitters(H, G, P, T, kind=0)
    def largest_cost(sp):
        worst = 0
        for g in range(int(sp.max()) + 1):
            n, r = int(H[sp == g].sum()), int(G[sp == g].sum())
            worst = max(worst, n * oracle.log2_q16(n) + ((T * n + r) << 16))
        return worst
    assert largest_cost(sp_c) == best_c
    assert largest_cost(sp_h) > best_c
    assert (sp_c != sp_h).any()


# ------------------------------------------------------------------ phase 4: windows


def test_windows_match_searchsorted():
    rng = np.random.default_rng(8)
    R = tuples(rng.integers(0, 300, 500, dtype=np.uint64))
    Rs, run_off = oracle.sort_runs(R, 5)
    S = tuples(np.sort(rng.integers(0, 320, 400, dtype=np.uint64)))
    tile_off = np.array([0, 1, 50, 128, 300, 400], dtype=np.uint64)
    win = oracle.windows(S, tile_off, Rs, run_off)
    for t in range(len(tile_off) - 1):
        lo_k, hi_k = S[int(tile_off[t]), 0], S[int(tile_off[t + 1]) - 1, 0]
        for j in range(5):
            run = Rs[int(run_off[j]):int(run_off[j + 1]), 0]
            assert win[t, j, 0] == np.searchsorted(run, lo_k, side="left")
            assert win[t, j, 1] == np.searchsorted(run, hi_k, side="right")
