"""Pins of the FP64 learned-model oracle (oracle/rmi.py) to things other than itself:
central finite differences, closed forms of the initial model and of Adam's first
step, torch's autograd and Adam (library routines), and least squares on exact lines."""
import numpy as np
import pytest

from oracle import rmi


def random_theta(seed):
    rng = np.random.default_rng(seed)
    th = rng.normal(0.0, 0.5, rmi.NPARAM)
    th[rmi.O_W1:rmi.O_B1] = rng.uniform(0.5, 2.0, rmi.H) * rng.choice([-1, 1], rmi.H)
    th[rmi.O_B1:rmi.O_W2] = rng.uniform(-1.0, 1.0, rmi.H)
    return th


def away_from_kinks(th, x, margin=1e-4):
    W1, b1, W2, b2, _, _ = rmi.unpack(th)
    a1 = np.outer(x, W1) + b1
    a2 = np.maximum(a1, 0) @ W2.T + b2
    return np.abs(a1).min() > margin and np.abs(a2).min() > margin


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    for seed in range(20):
        th = random_theta(seed)
        x = rng.uniform(0, 1, 24)
        y = rng.uniform(0, 1, 24)
        if not away_from_kinks(th, x):
            continue
        _, g = rmi.loss_grad(th, x, y)
        h = 1e-6
        fd = np.empty(rmi.NPARAM)
        for i in range(rmi.NPARAM):
            e = np.zeros(rmi.NPARAM)
            e[i] = h
            fd[i] = (rmi.loss_grad(th + e, x, y)[0] - rmi.loss_grad(th - e, x, y)[0]) / (2 * h)
        np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-8)
        return
    pytest.fail("no seed gave a kink-free batch")


def test_gradient_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    th = random_theta(3)
    x = rng.uniform(0, 1, 300)
    y = np.sort(rng.uniform(0, 1, 300))
    loss, g = rmi.loss_grad(th, x, y)
    t = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    W1, b1 = t[rmi.O_W1:rmi.O_B1], t[rmi.O_B1:rmi.O_W2]
    W2, b2 = t[rmi.O_W2:rmi.O_B2].reshape(32, 32), t[rmi.O_B2:rmi.O_W3]
    W3, b3 = t[rmi.O_W3:rmi.O_B3], t[rmi.O_B3]
    xt = torch.tensor(x, dtype=torch.float64)
    h1 = torch.relu(xt[:, None] * W1 + b1)
    h2 = torch.relu(torch.nn.functional.linear(h1, W2, b2))
    yh = h2 @ W3 + b3
    L = torch.mean((yh - torch.tensor(y, dtype=torch.float64)) ** 2)
    L.backward()
    assert abs(L.item() - loss) < 1e-12
    np.testing.assert_allclose(g, t.grad.numpy(), rtol=1e-10, atol=1e-14)


def test_initial_model_is_the_identity_cdf():
    x = np.linspace(0, 1, 101)
    np.testing.assert_allclose(rmi.forward(rmi.initial_theta(), x), x, atol=1e-15)
    loss, g = rmi.loss_grad(rmi.initial_theta(), x, x)
    assert loss == 0.0 and np.all(g == 0.0)


def test_first_adam_step_moves_each_weight_by_lr_times_sign():
    rng = np.random.default_rng(2)
    th = rng.normal(size=rmi.NPARAM)
    g = rng.normal(size=rmi.NPARAM)
    new, m, v = rmi.adam_step(th, np.zeros(rmi.NPARAM), np.zeros(rmi.NPARAM), g, 1, 0.01)
    np.testing.assert_allclose(th - new, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_adam_matches_torch_adam():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    th = rng.normal(size=rmi.NPARAM)
    grads = [rng.normal(size=rmi.NPARAM) for _ in range(6)]
    m = np.zeros(rmi.NPARAM)
    v = np.zeros(rmi.NPARAM)
    ours = th.copy()
    for t, g in enumerate(grads, start=1):
        ours, m, v = rmi.adam_step(ours, m, v, g, t, 3e-3)
    p = torch.nn.Parameter(torch.tensor(th, dtype=torch.float64))
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    for g in grads:
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
    np.testing.assert_allclose(ours, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_leaves_recover_exact_lines_and_match_polyfit():
    rng = np.random.default_rng(4)
    nleaf = 8
    keys = np.sort(rng.choice(np.arange(10**12, 10**12 + 10**7, dtype=np.uint64), 4000, replace=False))
    leaf = (np.arange(4000) * nleaf // 4000).astype(np.int64)
    slope = rng.uniform(1e-7, 1e-6, nleaf)
    icpt = rng.uniform(0, 1, nleaf)
    base = np.array([keys[leaf == l].min() for l in range(nleaf)], dtype=np.uint64)
    y = slope[leaf] * (keys - base[leaf]).astype(np.float64) + icpt[leaf]
    b0, a, b, cnt = rmi.fit_leaves(keys, y, leaf, nleaf)
    assert (b0 == base).all() and (cnt == 500).all()
    np.testing.assert_allclose(a, slope, rtol=1e-9)
    np.testing.assert_allclose(b, icpt, rtol=1e-9, atol=1e-12)
    noisy = y + rng.normal(0, 1e-3, y.shape)
    _, a2, b2, _ = rmi.fit_leaves(keys, noisy, leaf, nleaf)
    for l in range(nleaf):
        d = (keys[leaf == l] - base[l]).astype(np.float64)
        pa, pb = np.polyfit(d, noisy[leaf == l], 1)
        assert abs(pa - a2[l]) <= 1e-9 * abs(pa) + 1e-15 and abs(pb - b2[l]) < 1e-9


def test_leaf_edge_cases():
    keys = np.array([5, 5, 5, 9], dtype=np.uint64)
    y = np.array([0.1, 0.2, 0.3, 0.9])
    leaf = np.array([0, 0, 0, 2])
    base, a, b, cnt = rmi.fit_leaves(keys, y, leaf, 4)
    assert list(cnt) == [3, 0, 1, 0]
    assert a[0] == 0 and abs(b[0] - 0.2) < 1e-15 and base[0] == 5
    assert base[1] == 0 and a[1] == 0 and b[1] == (1 + 0.5) / 4
    assert a[2] == 0 and b[2] == 0.9
    # signed offsets below a leaf's base
    p = rmi.leaf_predict(np.array([3, 7], dtype=np.uint64), np.array([0, 0]), np.array([5], dtype=np.uint64),
                         np.array([0.5]), np.array([1.0]))
    assert list(p) == [0.0, 2.0]


def test_training_lowers_the_loss_on_a_skewed_cdf():
    import gen

    w = gen.zipf(1 << 14, 1 << 16, 0.9, seed=3)
    k = np.sort(w.s_host()[:, 0])
    idx = np.linspace(0, len(k) - 1, 2048).astype(np.int64)
    x = (k[idx] - k[0]).astype(np.float64) / float(k[-1] - k[0])
    y = (idx + 0.5) / len(k)
    th, hist = rmi.train(rmi.initial_theta(), x, y, 100, 3e-3)
    final = rmi.loss_grad(th, x, y)[0]
    assert final < 0.5 * hist[0]
