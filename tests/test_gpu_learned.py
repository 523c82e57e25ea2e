"""The learned CDF model on the GPU: gradients, Adam steps, tabulation and leaves
against the FP64 oracle (oracle/rmi.py); learned joins bit-identical to the
oracle and to the plain modes; and what the trained network gains."""
import numpy as np
import pytest

import gen
import oracle
from oracle import rmi
from helpers import to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1207_0145_gb300 import Plan, mpsm as M  # noqa: E402


def f32(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def random_theta(seed):
    rng = np.random.default_rng(seed)
    th = rng.normal(0.0, 0.3, rmi.NPARAM)
    th[rmi.O_W1:rmi.O_B1] = rng.uniform(0.5, 2.0, rmi.H) * rng.choice([-1, 1], rmi.H)
    th[rmi.O_B1:rmi.O_W2] = rng.uniform(-1.0, 1.0, rmi.H)
    return th.astype(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def plan():
    with Plan(1 << 22, 1 << 22) as p:  # fit capacity (1/64 of the sides) >= 65536 points
        yield p


@pytest.mark.parametrize("n,seed", [(4096, 1), (300, 2), (33, 3), (1, 4)])
def test_gradient_matches_fp64_oracle(plan, n, seed):
    rng = np.random.default_rng(seed)
    th = random_theta(seed)
    x = rng.uniform(0, 1, n).astype(np.float32).astype(np.float64)
    y = np.sort(rng.uniform(0, 1, n)).astype(np.float32).astype(np.float64)
    loss, g = plan.rmi_loss_grad(f32(x), f32(y), f32(th))
    want_loss, want_g = rmi.loss_grad(th, x, y)
    assert abs(loss - want_loss) <= 1e-4 * abs(want_loss) + 1e-6
    np.testing.assert_allclose(g.cpu().numpy(), want_g, rtol=1e-4, atol=1e-6)


def test_adam_steps_track_the_oracle(plan):
    w = gen.zipf(1 << 14, 1 << 16, 0.9, seed=5)
    k = np.sort(w.s_host()[:, 0])
    idx = np.linspace(0, len(k) - 1, 4096).astype(np.int64)
    x = ((k[idx] - k[0]).astype(np.float64) / float(k[-1] - k[0])).astype(np.float32).astype(np.float64)
    y = ((idx + 0.5) / len(k)).astype(np.float32).astype(np.float64)
    th0 = rmi.initial_theta()
    theta = f32(th0)
    losses = plan.rmi_train(f32(x), f32(y), theta, 10, 3e-3)
    want, hist = rmi.train(th0, x, y, 10, 3e-3)
    np.testing.assert_allclose(losses, hist, rtol=1e-3)
    d = np.abs(theta.cpu().numpy() - want)
    assert np.median(d) < 1e-6 and d.max() < 2 * 10 * 3e-3


def fit_case(plan, keys, steps=200):
    k = np.sort(keys.astype(np.uint64))
    y = ((np.arange(len(k)) + 0.5) / len(k)).astype(np.float32)
    kt = to_dev(k.view(np.int64))
    plan.rmi_fit(kt, f32(y), int(k[0]), int(k[-1]), steps, 3e-3)
    return k, y.astype(np.float64), kt, plan.rmi_export(0)


@pytest.mark.parametrize("case", ["uniform", "zipf", "sparse"])
def test_tabulation_and_leaves_match_the_oracle(plan, case):
    if case == "uniform":
        keys = gen.plain(1 << 15, 1 << 15, seed=7).r_host()[:, 0]
    elif case == "zipf":
        keys = gen.zipf(1 << 14, 1 << 16, 0.9, seed=8).s_host()[:, 0]
    else:
        keys = gen.sparse(1 << 16, 16, seed=9).r_host()[:, 0]
    k, y, kt, m = fit_case(plan, keys)
    assert m["fit_n"] == len(k) and m["train_n"] == min(len(k), 4096)
    # tabulated root: the oracle's forward pass (FP64) at every cell centre, with the GPU's weights
    th = m["theta"].astype(np.float64)
    rng_ = int(m["kmax"]) - int(m["kmin"])
    c = np.arange(m["ncell"], dtype=np.float64)
    mid = np.minimum(c * 2.0 ** m["cshift"] + (2 ** m["cshift"] // 2), rng_)
    f = rmi.forward(th, (mid / rng_).astype(np.float32).astype(np.float64) if rng_ else 0 * mid) * 4096
    sure = np.abs(f - np.round(f)) > 1e-2
    want_leaf = np.clip(np.floor(f), 0, 4095).astype(np.int64)
    got_leaf = m["cell_leaf"][: m["ncell"]].astype(np.int64)
    assert (got_leaf[sure] == want_leaf[sure]).all()
    # leaves: the oracle's least squares under the GPU's routing
    cell = np.minimum((k - np.uint64(m["kmin"])) >> np.uint64(m["cshift"]), m["ncell"] - 1).astype(np.int64)
    leaf = m["cell_leaf"][cell].astype(np.int64)
    base, a, b, cnt = rmi.fit_leaves(k, y, leaf, 4096)
    used = cnt > 0
    assert (m["leaf_base"][used] == base[used]).all()
    want = rmi.leaf_predict(k, leaf, base, a, b)
    got = rmi.leaf_predict(k, leaf, m["leaf_base"], m["leaf_a"].astype(np.float64), m["leaf_b"].astype(np.float64))
    assert np.abs(got - want).max() < 2e-5
    # inference kernel == the stage-2 formula with the exported tables
    yh, lf = plan.rmi_predict(kt)
    assert (lf.cpu().numpy() == leaf).all()
    np.testing.assert_allclose(yh.cpu().numpy(), np.clip(got, 0, 1), atol=2e-6)


def join_all(p, w):
    R, S = to_dev(w.r_host().view(np.int64)), to_dev(w.s_host().view(np.int64))
    return p.join(R, S), p.stats()


def workloads():
    return [gen.plain(70_000, 300_000, seed=11), gen.zipf(50_000, 400_000, 0.9, seed=12),
            gen.sparse(60_000, 90_000, seed=13), gen.zipf(3000, 200_000, 1.1, seed=14),
            gen.plain(1, 1000, seed=15), gen.plain(20_000, 1, seed=16)]


@pytest.mark.parametrize("split,search", [(1, 0), (0, 1), (1, 1)])
def test_learned_joins_are_exact(split, search):
    ws = workloads()
    with Plan(1 << 17, 1 << 19, splitter_mode=split, search_mode=search) as p, Plan(1 << 17, 1 << 19) as q:
        for w in ws:
            got, st = join_all(p, w)
            want = oracle.join(w.r_host(), w.s_host())
            assert got == want, (w, got, want)
            assert got == join_all(q, w)[0]
            assert got == p.join(to_dev(w.r_host().view(np.int64)), to_dev(w.s_host().view(np.int64)))


def test_learned_edge_keys_and_duplicates():
    rng = np.random.default_rng(3)
    R = np.zeros((5000, 2), dtype=np.uint64)
    R[:, 0] = rng.choice(np.array([0, 1, 2**63, 2**64 - 2, 2**64 - 1], dtype=np.uint64), 5000)
    R[:, 1] = rng.integers(0, 2**63, 5000, dtype=np.uint64)
    S = np.zeros((20000, 2), dtype=np.uint64)
    S[:, 0] = rng.choice(np.array([0, 1, 5, 2**63, 2**64 - 1], dtype=np.uint64), 20000)
    S[:, 1] = rng.integers(0, 2**63, 20000, dtype=np.uint64)
    with Plan(1 << 14, 1 << 16, splitter_mode=1, search_mode=1, partitions_s=64) as p:
        got = p.join(to_dev(R.view(np.int64)), to_dev(S.view(np.int64)))
    assert got == oracle.join(R, S)


def test_learned_splitters_balance_a_zipf_skew():
    """Hot keys of Zipf(0.9) make equal-width fine buckets unbalanced; the learned
    quantile boundaries with hot-key spreading keep partitions near the mean."""
    w = gen.zipf(1 << 18, 1 << 21, 0.9, seed=21)
    with Plan(1 << 18, 1 << 21, partitions_s=256) as h, \
            Plan(1 << 18, 1 << 21, partitions_s=256, splitter_mode=1) as l:
        a, sa = join_all(h, w)
        b, sb = join_all(l, w)
    assert a == b
    # the cost-balanced histogram splitters cannot split the hot fine bucket: they
    # fall back to fewer, larger partitions; the learned ones keep all 256 near the mean
    assert sb["partitions_s"] == 256 and sb["imbalance"] < 1.5, sb
    assert sb["part_max"] * 4 < sa["part_max"], (sa["part_max"], sb["part_max"])


@pytest.mark.parametrize("case", ["zipf", "sparse"])
def test_training_lowers_prediction_error(case):
    """What the trained network gains: against the same pipeline after one Adam step
    (still the initial identity CDF), training lowers the root's loss on both sides;
    and its predictions find a key's partition among P = 256 boundaries in fewer
    probes than the 8 a binary search of the boundaries takes."""
    w = gen.zipf(1 << 17, 1 << 20, 0.9, seed=22) if case == "zipf" else gen.sparse(1 << 18, 1 << 18, seed=23)
    res = {}
    for steps in (1, 200):
        with Plan(w.n_r, w.n_s, splitter_mode=1, search_mode=1, learn_steps=steps, partitions_s=256) as p:
            res[steps] = join_all(p, w)
    assert res[1][0] == res[200][0]
    s1, s200 = res[1][1], res[200][1]
    assert s200["loss_s"] < 0.5 * s1["loss_s"]
    if case == "sparse":  # uniform R keys (zipf case) already have the identity CDF
        assert s200["loss_r"] < 0.5 * s1["loss_r"]
    assert s200["part_probes"] < 8.0 and s200["part_probes"] <= 1.05 * s1["part_probes"], (s1, s200)
