"""Role reversal (partition R and cut S into runs, or partition the smaller input):
the same count, checksum and pairs as the default roles and the oracle."""
import numpy as np
import pytest

import gen
import oracle
from helpers import to_dev, sort_tuples

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_0145_gb300 import Plan, mpsm as M  # noqa: E402


def cases():
    rng = np.random.default_rng(5)
    out = [gen.plain(60_000, 240_000, seed=1), gen.plain(300_000, 50_000, seed=2), gen.zipf(40_000, 160_000, 0.9, seed=3),
           gen.sparse(50_000, 70_000, seed=4), gen.plain(1, 999, seed=5), gen.plain(999, 1, seed=6)]
    out = [(w.r_host(), w.s_host()) for w in out]
    R = np.zeros((7000, 2), dtype=np.uint64)
    S = np.zeros((9000, 2), dtype=np.uint64)
    R[:, 0] = rng.integers(0, 50, 7000, dtype=np.uint64)
    S[:, 0] = rng.integers(0, 50, 9000, dtype=np.uint64)
    R[:, 1] = rng.integers(0, 2**64 - 1, 7000, dtype=np.uint64)
    S[:, 1] = rng.integers(0, 2**64 - 1, 9000, dtype=np.uint64)
    out.append((R, S))
    return out


@pytest.mark.parametrize("side", [M.PART_R, M.PART_SMALLER])
def test_reversed_roles_give_the_same_join(side):
    with Plan(1 << 19, 1 << 19, partition_side=side) as p:
        for R, S in cases():
            assert p.join(to_dev(R), to_dev(S)) == oracle.join(R, S)


def test_reversed_roles_keep_the_pair_order():
    w = gen.zipf(20_000, 50_000, 0.8, seed=9)
    R, S = w.r_host(), w.s_host()
    cnt, _, want = oracle.join(R, S, with_pairs=True)
    outs = []
    for side in (M.PART_S, M.PART_R):
        with Plan(w.n_r, w.n_s, partition_side=side) as p:
            buf = torch.empty((cnt, 2), dtype=torch.int64, device="cuda")
            assert p.join(to_dev(R), to_dev(S), pairs=buf)[0] == cnt
            outs.append(sort_tuples(buf.cpu().numpy().view(np.uint64)))
    assert (outs[0] == outs[1]).all()
    assert (outs[0] == sort_tuples(np.asarray(want, dtype=np.uint64))).all()


def test_reversed_roles_through_host_buffers():
    w = gen.plain(30_000, 90_000, seed=11)
    R, S = w.r_host(), w.s_host()
    Rh = torch.from_numpy(R.view(np.int64)).pin_memory()
    Sh = torch.from_numpy(S.view(np.int64)).pin_memory()
    with Plan(w.n_r, w.n_s, partition_side=M.PART_R) as p:
        assert p.join_host(Rh, Sh) == oracle.join(R, S)


def test_reversed_roles_report_pair_capacity_like_the_default():
    w = gen.plain(10_000, 40_000, seed=12)
    R, S = to_dev(w.r_host()), to_dev(w.s_host())
    for side in (M.PART_S, M.PART_R, M.PART_SMALLER):
        small = torch.zeros((100, 2), dtype=torch.int64, device="cuda")
        with Plan(w.n_r, w.n_s, partition_side=side) as p:
            with pytest.raises(M.MPSMError) as e:
                p.join(R, S, pairs=small)
        assert e.value.status == M.ERR_CAPACITY and "40000" in str(e.value)
        assert small.abs().sum().item() == 0

