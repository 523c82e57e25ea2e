"""Parity where the kernels take their deep paths, element by element.

- Sparse 64-bit keys (64 clusters over the whole u64 range) in large runs: R's run
  sort needs at least three radix levels and S's partition sort at least two; the
  sorted runs and partitions are compared with the oracle.
- The fused path (phases 3 and 4 in one kernel): every final S segment's window in
  every run against the oracle's lower and upper bounds for the segment's key
  bounds; the segments hold the kept S exactly once, each key inside its bounds.
- Materialised pairs at 10 Mi S tuples against the generator's per-row closed form
  (each foreign-key S row pairs with the R row it was drawn from).
"""
import numpy as np
import pytest

import gen
import oracle
from tests.helpers import from_dev_ptr, random_tuples, same_multiset, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_0145_gb300 import Plan  # noqa: E402

W_XS, W_Y = 3, 4


def test_sparse_deep_levels_runs_and_partitions():
    w = gen.sparse(1 << 21, 1 << 21, seed=71)
    R, S = w.r_host(), w.s_host()
    with Plan(w.n_r, w.n_s, runs_r=2) as p:
        dR, dS = to_dev(R), to_dev(S)
        p.sort_runs(dR)
        v = p.view()
        got = from_dev_ptr(v.r_runs, len(R))
        off = from_dev_ptr(v.run_offsets, 3, width=1)
        want, want_off = oracle.sort_runs(R, 2)
        assert (off == want_off).all()
        assert (got == want).all()  # unique keys: the sorted runs are unique
        p.splitters(dS)
        p.scatter()
        p.sort_partitions()
        st = p.stats()
        assert st["levels_r"] >= 3 and st["levels_s"] >= 2, (st["levels_r"], st["levels_s"])
        v = p.view()
        kept = S[(S[:, 0] >= np.uint64(v.key_min)) & (S[:, 0] <= np.uint64(v.key_max))]
        got_s = from_dev_ptr(v.s_buffer, v.s_kept)
        assert v.s_kept == len(kept)
        assert (got_s[:, 0] == np.sort(kept[:, 0])).all()
        assert same_multiset(got_s, kept)
        p.search()
        assert p.merge_join() == oracle.join(R, S) == oracle.closed_form(w)


# runs of 32K tuples (the automatic count) put every fence of a run in the search's
# shared-memory top level; runs of 512K and 350K tuples make it every 4th and 3rd one
@pytest.mark.parametrize("w,runs", [(gen.sparse(1 << 20, 1 << 21, seed=72), 0), (gen.plain(1 << 20, 1 << 22, seed=73), 0),
                                    (gen.zipf(1 << 19, 1 << 21, 1.1, seed=74), 0),
                                    (gen.plain(1 << 20, 1 << 22, seed=76), 2), (gen.sparse(1 << 20, 1 << 21, seed=77), 3)])
def test_fused_segment_windows_match_oracle(w, runs):
    R, S = w.r_host(), w.s_host()
    with Plan(w.n_r, w.n_s, runs_r=runs) as p:
        assert p.join(to_dev(R), to_dev(S)) == oracle.join(R, S)
        v = p.view()
        T = v.runs_r
        Rs = from_dev_ptr(v.r_runs, len(R))
        run_off = from_dev_ptr(v.run_offsets, T + 1, width=1)
        n = v.n_segments
        segs = from_dev_ptr(v.segments, n, width=5)  # offset, length, key_lo, key_hi, job | flags << 32
        where = (segs[:, 4] >> np.uint64(32)) & np.uint64(7)
        assert set(np.unique(where).tolist()) <= {W_XS, W_Y}
        # the oracle's windows: a two-key "tile" per segment holding its bounds
        Ss = np.zeros((2 * n, 2), dtype=np.uint64)
        Ss[0::2, 0] = segs[:, 2]
        Ss[1::2, 0] = segs[:, 3]
        want = oracle.windows(Ss, np.arange(0, 2 * n + 1, 2, dtype=np.uint64), Rs, run_off)
        got = from_dev_ptr(v.seg_windows, n * v.window_stride * 2, width=1, dtype=np.uint32)
        got = got.reshape(n, v.window_stride, 2)[:, :T, :].astype(np.uint64)
        assert (got == want).all()
        # every kept S tuple in exactly one segment, inside that segment's bounds
        kept = S[(S[:, 0] >= np.uint64(v.key_min)) & (S[:, 0] <= np.uint64(v.key_max))]
        size = max(int((segs[:, 0] + segs[:, 1]).max()), 1)
        bufs = {W_XS: from_dev_ptr(v.s_buffer, size), W_Y: from_dev_ptr(v.pass_buffer, size)}
        parts = []
        for (o, ln, lo, hi, _), wh in zip(segs.tolist(), where.tolist()):
            t = bufs[wh][o:o + ln]
            assert ((t[:, 0] >= np.uint64(lo)) & (t[:, 0] <= np.uint64(hi))).all()
            parts.append(t)
        assert same_multiset(np.concatenate(parts), kept)


def test_pairs_at_ten_million_match_the_per_row_closed_form():
    w = gen.plain(1 << 22, 10 << 20, seed=75)
    R, S = w.r_host(), w.s_host()
    rows = w.s_rows_host().astype(np.int64)
    want = np.stack([R[rows, 1], S[:, 1]], axis=1)  # (r_payload, s_payload) of every S row
    out = torch.empty((w.n_s, 2), dtype=torch.int64, device="cuda")
    with Plan(w.n_r, w.n_s) as p:
        assert p.join(to_dev(R), to_dev(S), pairs=out) == oracle.closed_form(w)
    assert same_multiset(out.cpu().numpy().view(np.uint64), want)


def test_hot_key_in_both_inputs_on_the_fused_path():
    # half of R is one key and 20000 S tuples carry it: the S key's constant segments
    # (in 8192-tuple pieces) meet a window of about 2^18 R tuples in each of the 4 runs,
    # which every thread of the block shares
    rng = np.random.default_rng(97)
    R = random_tuples(rng, 1 << 21, 1 << 30)
    S = random_tuples(rng, 1 << 21, 1 << 30)
    R[: 1 << 20, 0] = np.uint64(7)
    S[:20000, 0] = np.uint64(7)
    R = R[rng.permutation(len(R))]
    with Plan(len(R), len(S), runs_r=4) as p:
        assert p.join(to_dev(R), to_dev(S)) == oracle.join(R, S)
        assert p.device_errors() == 0
