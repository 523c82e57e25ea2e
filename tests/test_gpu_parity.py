"""GPU parity: every phase of the CUDA path against the CPU oracle, element by element.

Integer work is compared bit-exactly.  Where the method leaves an order open
(tuples inside a chunk's sub-partition after the scatter, equal keys after a
sort, the order of output pairs) the unique part is compared exactly and the
rest as multisets.
"""
import numpy as np
import pytest

import gen
import oracle
from tests.helpers import from_dev_ptr, random_tuples, same_multiset, sort_tuples, to_dev, U64

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_0145_gb300 import MPSMError, Plan  # noqa: E402
from paper_1207_0145_gb300 import mpsm as M  # noqa: E402


def join_gpu(R, S, **opt):
    with Plan(max(len(R), 1), max(len(S), 1), **opt) as p:
        return p.join(to_dev(R), to_dev(S))


# ------------------------------------------------------------------ whole join


def test_config_plain_1M_4M_matches_oracle_and_closed_form():
    w = gen.CONFIGS["plain-1M-4M"]()
    R, S = w.r_host(), w.s_host()
    want = oracle.join(R, S)
    assert want[0] == 4 * (1 << 20)
    assert oracle.closed_form(w) == want
    assert join_gpu(R, S, runs_r=32) == want


@pytest.mark.parametrize("case", range(24))
def test_random_joins_match_oracle(case):
    rng = np.random.default_rng(1000 + case)
    nr = int(rng.choice([1, 7, 100, 5000, 20000, 70000]))
    ns = int(rng.choice([1, 9, 300, 8000, 50000, 150000]))
    domain = int(rng.choice([1, 3, 100, 10_000, 1 << 32, 1 << 64]))
    R = random_tuples(rng, nr, domain, extremes=bool(case % 3 == 0))
    S = random_tuples(rng, ns, domain, extremes=bool(case % 4 == 0))
    opt = dict(runs_r=int(rng.choice([0, 1, 3, 32, 100])), partitions_s=int(rng.choice([0, 1, 2, 7, 64])),
               fine_bits=int(rng.choice([0, 1, 4, 12])), radix_bits=int(rng.choice([0, 4, 8, 11])),
               join_tile=int(rng.choice([0, 256, 1024])))
    assert join_gpu(R, S, **opt) == oracle.join(R, S), opt


@pytest.mark.parametrize("w", [gen.zipf(300_000, 1_200_000, 0.9, seed=3), gen.sparse(200_000, 200_000, seed=4),
                               gen.zipf(50_000, 800_000, 1.2, seed=5)])
def test_skewed_and_sparse_workloads(w):
    R, S = w.r_host(), w.s_host()
    want = oracle.join(R, S)
    assert want == oracle.closed_form(w)
    assert join_gpu(R, S) == want
    assert join_gpu(R, S, runs_r=7, partitions_s=5, fine_bits=6) == want


def test_edge_cases():
    e = np.zeros((0, 2), dtype=np.uint64)
    one = np.array([[5, 9]], dtype=np.uint64)
    assert join_gpu(e, e) == (0, 0)
    assert join_gpu(one, e) == (0, 0)
    assert join_gpu(e, one) == (0, 0)
    assert join_gpu(one, one) == (1, 18)
    # all keys equal on both sides: every pair matches (M:N, groups straddle tiles and runs)
    R = np.stack([np.full(3000, 77, np.uint64), np.arange(3000, dtype=np.uint64)], 1)
    S = np.stack([np.full(20000, 77, np.uint64), np.arange(20000, dtype=np.uint64) * 3], 1)
    assert join_gpu(R, S) == oracle.join(R, S) == (3000 * 20000, (20000 * sum(range(3000)) + 3000 * 3 * sum(range(20000))) % (1 << 64))
    # extreme keys only
    R = np.array([[0, 1], [U64, 2], [U64, 3]], dtype=np.uint64)
    S = np.array([[U64, 10], [0, 20], [U64 - 1, 30]], dtype=np.uint64)
    assert join_gpu(R, S) == oracle.join(R, S)
    # disjoint key ranges: everything in S is dropped before partitioning
    rng = np.random.default_rng(2)
    R = random_tuples(rng, 10000, 1000)
    S = random_tuples(rng, 10000, 1000)
    S[:, 0] += np.uint64(5000)
    assert join_gpu(R, S) == (0, 0)
    # heavy duplicates in R and S with a tile-sized hot key
    R = random_tuples(rng, 40000, 50)
    S = random_tuples(rng, 100000, 60)
    assert join_gpu(R, S, join_tile=256) == oracle.join(R, S)


def test_runs_straddling_smem_capacity():
    """Runs just above/below the in-SMEM capacity and keys spread over 64 bits."""
    rng = np.random.default_rng(9)
    for nr in (8191, 8192, 8193, 16385, 3 * 8192 + 5):
        R = random_tuples(rng, nr, 1 << 64)
        S = np.concatenate([R[rng.integers(0, nr, 20000)], random_tuples(rng, 5000, 1 << 64)])
        S[:, 1] = rng.integers(0, U64, len(S), dtype=np.uint64, endpoint=True)
        assert join_gpu(R, S, runs_r=1) == oracle.join(R, S), nr


def test_deterministic_results():
    w = gen.zipf(100_000, 400_000, 0.9, seed=8)
    R, S = to_dev(w.r_host()), to_dev(w.s_host())
    with Plan(len(R), len(S)) as p:
        a = p.join(R, S)
        b = p.join(R, S)
    assert a == b


# ------------------------------------------------------------------ phase by phase


def run_phases(R, S, **opt):
    p = Plan(len(R), len(S), **opt)
    dR, dS = to_dev(R), to_dev(S)
    return p, dR, dS


def test_phase1_sorted_runs_match_oracle():
    w = gen.plain(300_000, 10, seed=11)
    R = w.r_host()
    for T in (1, 5, 32):
        p, dR, _ = run_phases(R, R[:1], runs_r=T)
        p.sort_runs(dR)
        v = p.view()
        got = from_dev_ptr(v.r_runs, len(R))
        off = from_dev_ptr(v.run_offsets, T + 1, width=1)
        want, want_off = oracle.sort_runs(R, T)
        assert (off == want_off).all()
        assert (got == want).all()  # unique keys: the sorted run is unique
        p.close()


def test_phase1_runs_with_duplicate_keys():
    rng = np.random.default_rng(12)
    R = random_tuples(rng, 100_000, 500)
    p, dR, _ = run_phases(R, R[:1], runs_r=6)
    p.sort_runs(dR)
    v = p.view()
    got = from_dev_ptr(v.r_runs, len(R))
    want, off = oracle.sort_runs(R, 6)
    assert (got[:, 0] == want[:, 0]).all()
    for j in range(6):
        a, b = int(off[j]), int(off[j + 1])
        assert same_multiset(got[a:b], want[a:b])
    p.close()


def phase2_oracle(R, S, v, T):
    """The oracle's phase 2 for the library's chunking (workers) and parameters."""
    Rs, run_off = oracle.sort_runs(R, T)
    kmin, kmax = int(Rs[:, 0].min()), int(Rs[:, 0].max())
    return Rs, run_off, kmin, kmax


# (8, 200) and (12, 2000): few buckets per partition, so the splitter solve reaches its
# candidate bisection early; (12, 512): the headline's partition count
@pytest.mark.parametrize("fine_bits,parts,kind", [(12, 0, 0), (6, 9, 0), (2, 2, 0), (10, 0, 1), (12, 0, 1),
                                                  (10, 0, 0), (8, 200, 0), (12, 2000, 0), (12, 512, 0)])
def test_phase2_histograms_splitters_prefix_sums(fine_bits, parts, kind):
    # kind 1: equi-height splitters (Sec. 5.6) on the negatively correlated workload
    w = gen.zipf(60_000, 500_000, 0.9, seed=13) if (kind == 0 and fine_bits != 10) else gen.negcorr(60_000, 240_000, seed=17)
    R, S = w.r_host(), w.s_host()
    T = 8
    mode = M.SPLIT_EQUI_HEIGHT if kind else M.SPLIT_HIST
    p, dR, dS = run_phases(R, S, runs_r=T, fine_bits=fine_bits, partitions_s=parts, splitter_mode=mode)
    p.sort_runs(dR)
    p.splitters(dS)
    v = p.view()
    Rs, run_off, kmin, kmax = phase2_oracle(R, S, v, T)
    assert (v.key_min, v.key_max) == (kmin, kmax)
    nb, shift = oracle.fine_geometry(kmin, kmax, fine_bits or 12)
    assert (v.nfine, v.fine_shift) == (nb, shift)
    chunk_off = from_dev_ptr(v.s_chunk_offsets, v.s_chunks + 1, width=1)
    assert chunk_off[0] == 0 and chunk_off[-1] == len(S)
    h = oracle.worker_histograms(S, chunk_off, kmin, kmax, shift, nb)
    H = h.sum(axis=0)
    assert (from_dev_ptr(v.fine_s, nb, width=1) == H).all()
    G = oracle.run_counts(Rs, run_off, kmin, kmax, shift, nb)
    assert (from_dev_ptr(v.fine_r, nb, width=1) == G).all()
    P_req = parts or 32
    sp, nparts, _ = oracle.splitters(H, G, min(P_req, nb), T, kind=kind)
    assert v.partitions_s == nparts
    assert (from_dev_ptr(v.splitters, nb, width=1, dtype=np.uint32) == sp).all()
    # per-worker partition histograms and prefix sums (the ps equation under Fig. 6)
    hp = np.zeros((v.s_chunks, nparts), dtype=np.uint64)
    for f in range(nb):
        hp[:, sp[f]] += h[:, f]
    ps, part_off = oracle.prefix_sums(hp)
    got_ps = from_dev_ptr(v.chunk_offsets, v.s_chunks * nparts, width=1, dtype=np.uint32).reshape(v.s_chunks, nparts)
    assert (got_ps.astype(np.uint64) == ps).all()
    assert (from_dev_ptr(v.part_offsets, nparts + 1, width=1) == part_off).all()
    # scatter: every worker's sub-partition holds exactly its tuples (order inside is free)
    p.scatter()
    v = p.view()
    got = from_dev_ptr(v.s_buffer, int(part_off[-1]))
    want = oracle.scatter(S, chunk_off, kmin, kmax, shift, sp, ps)
    assert v.s_kept == len(want)
    for i in range(v.s_chunks):
        for j in range(nparts):
            a = int(ps[i, j])
            b = a + int(hp[i, j])
            assert same_multiset(got[a:b], want[a:b]), (i, j)
    p.close()


@pytest.mark.parametrize("w,search", [(gen.plain(200_000, 900_000, seed=14), 0), (gen.sparse(100_000, 300_000, seed=15), 0),
                                      (gen.zipf(100_000, 700_000, 1.1, seed=16), 0),
                                      (gen.plain(200_000, 900_000, seed=14), 2), (gen.sparse(100_000, 300_000, seed=15), 2),
                                      (gen.zipf(100_000, 700_000, 1.1, seed=16), 2), (gen.locskew(150_000, 500_000, seed=18), 2)])
def test_phase3_sorted_partitions_and_phase4(w, search):
    # search 2: merge starts by interpolation search (Sec. 3.2.2); the windows are exact either way
    R, S = w.r_host(), w.s_host()
    T = 16
    p, dR, dS = run_phases(R, S, runs_r=T, join_tile=1024, search_mode=search)
    p.sort_runs(dR)
    p.splitters(dS)
    p.scatter()
    p.sort_partitions()
    v = p.view()
    kmin, kmax = v.key_min, v.key_max
    kept = S[(S[:, 0] >= np.uint64(kmin)) & (S[:, 0] <= np.uint64(kmax))]
    got = from_dev_ptr(v.s_buffer, v.s_kept)
    assert v.s_kept == len(kept)
    assert (got[:, 0] == np.sort(kept[:, 0])).all()
    assert same_multiset(got, kept)
    # search windows vs the oracle's lower/upper bounds
    p.search()
    v = p.view()
    tile = v.join_tile
    tile_off = np.minimum(np.arange(v.tiles + 1, dtype=np.uint64) * np.uint64(tile), np.uint64(v.s_kept))
    Rs = from_dev_ptr(v.r_runs, len(R))
    run_off = from_dev_ptr(v.run_offsets, T + 1, width=1)
    want_win = oracle.windows(got, tile_off, Rs, run_off)
    got_win = from_dev_ptr(v.windows, v.tiles * T * 2, width=1, dtype=np.uint32).reshape(v.tiles, T, 2)
    assert (got_win.astype(np.uint64) == want_win).all()
    assert p.merge_join() == oracle.join(R, S)
    p.close()


@pytest.mark.parametrize("mode", [M.SPLIT_HIST, M.SPLIT_EQUI_HEIGHT, M.SPLIT_LEARNED])
def test_negatively_correlated_join_every_splitter_mode(mode):
    # Sec. 5.6 workload: the splitters change the partitions, never the result
    w = gen.negcorr(150_000, 600_000, seed=23)
    R, S = w.r_host(), w.s_host()
    want = oracle.join(R, S)
    assert want == oracle.closed_form(w)
    for side in (M.PART_S, M.PART_R):
        with Plan(w.n_r, w.n_s, splitter_mode=mode, fine_bits=10, partition_side=side) as p:
            assert p.join(to_dev(R), to_dev(S)) == want
            if mode == M.SPLIT_EQUI_HEIGHT and side == M.PART_S:
                assert p.stats()["imbalance"] < 1.5  # equal sizes up to the fine-bucket granularity


@pytest.mark.parametrize("w", [gen.plain(300_000, 1_200_000, seed=31), gen.zipf(100_000, 400_000, 0.9, seed=32),
                               gen.sparse(100_000, 200_000, seed=33), gen.locskew(200_000, 800_000, seed=34),
                               gen.negcorr(100_000, 400_000, seed=35)])
def test_interpolation_search_join(w):
    # the fused path's windows (every segment x run) and the step path's tile starts
    R, S = w.r_host(), w.s_host()
    want = oracle.join(R, S)
    for flags in (0, M.FLAG_UNFUSED):
        with Plan(w.n_r, w.n_s, search_mode=M.SEARCH_INTERP, flags=flags) as p:
            assert p.join(to_dev(R), to_dev(S)) == want


def test_interpolation_search_probes_on_uniform_runs():
    # on uniform keys the rule of proportion lands next to the answer: far fewer
    # probes than the binary search's log2 of the run length
    w = gen.plain(1 << 22, 1 << 22, seed=36)
    R, S = w.r_host(), w.s_host()
    probes = {}
    for mode in (M.SEARCH_BINARY, M.SEARCH_INTERP):
        with Plan(w.n_r, w.n_s, search_mode=mode, runs_r=4, flags=M.FLAG_UNFUSED) as p:
            assert p.join(to_dev(R), to_dev(S)) == oracle.closed_form(w)
            probes[mode] = p.stats()["search_probes"]
    assert probes[M.SEARCH_BINARY] >= 20  # log2 of a 2^20-tuple run
    assert probes[M.SEARCH_INTERP] < 10


def test_equi_height_with_more_partitions_requested_than_fine_buckets():
    w = gen.zipf(80_000, 300_000, 0.9, seed=37)
    R, S = w.r_host(), w.s_host()
    with Plan(w.n_r, w.n_s, splitter_mode=M.SPLIT_EQUI_HEIGHT, fine_bits=3, partitions_s=20) as p:
        assert p.join(to_dev(R), to_dev(S)) == oracle.join(R, S)
        assert 1 <= p.stats()["partitions_s"] <= 8


# ------------------------------------------------------------------ pairs


def test_materialised_pairs_match_oracle():
    rng = np.random.default_rng(21)
    R = random_tuples(rng, 20_000, 5_000)
    S = random_tuples(rng, 60_000, 5_000)
    c, k, want = oracle.join(R, S, with_pairs=True)
    out = torch.zeros((c, 2), dtype=torch.int64, device="cuda")
    with Plan(len(R), len(S), runs_r=5) as p:
        got = p.join(to_dev(R), to_dev(S), pairs=out)
    assert got == (c, k)
    pairs = out.cpu().numpy().view(np.uint64)
    assert (sort_tuples(pairs) == want).all()


def test_pairs_capacity_error_reports_needed_size():
    w = gen.plain(10_000, 40_000, seed=3)
    small = torch.zeros((100, 2), dtype=torch.int64, device="cuda")
    with Plan(10_000, 40_000) as p:
        with pytest.raises(MPSMError) as e:
            p.join(to_dev(w.r_host()), to_dev(w.s_host()), pairs=small)
    assert e.value.status == M.ERR_CAPACITY
    assert "40000" in str(e.value)
    assert small.abs().sum().item() == 0  # nothing written past the check


# ------------------------------------------------------------------ argument and state errors


def test_invalid_arguments_and_order_errors():
    import ctypes

    with Plan(1000, 1000) as p:
        R = torch.zeros((2000, 2), dtype=torch.int64, device="cuda")
        with pytest.raises(MPSMError) as e:
            p.join(R, R[:10])
        assert e.value.status == M.ERR_INVALID_ARG
        rc = M.lib().mpsm_join(p.handle, R.data_ptr() + 8, 10, R.data_ptr(), 10, ctypes.byref(ctypes.c_uint64()),
                               ctypes.byref(ctypes.c_uint64()), None)
        assert rc == M.ERR_INVALID_ARG  # misaligned
        q = Plan(100, 100)
        with pytest.raises(MPSMError) as e:
            q.scatter()
        assert e.value.status == M.ERR_STATE
        q.close()


# ------------------------------------------------------------------ batched


def test_batched_joins_match_per_job_oracle():
    rng = np.random.default_rng(31)
    jobs, want = [], []
    for i in range(12):
        nr = int(rng.integers(1, 60_000))
        w = gen.Workload(gen.KIND_ZIPF if i % 2 else gen.KIND_UNIFORM, nr, nr * int(rng.choice([1, 2, 4, 8])),
                         seed=500 + i, theta=0.8)
        R, S = w.r_host(), w.s_host()
        want.append(oracle.join(R, S))
        jobs.append((to_dev(R), to_dev(S)))
    tr = sum(len(r) for r, _ in jobs)
    ts = sum(len(s) for _, s in jobs)
    with Plan(tr, ts, max_jobs=len(jobs)) as p:
        c1, k1 = p.join_batch(jobs)
        c2, k2 = p.join_batch(jobs)  # graph replay
    assert list(zip(c1, k1)) == want
    assert (c1, k1) == (c2, k2)
