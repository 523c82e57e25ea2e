"""rmi.py -- FP64 reference of the learned CDF model (a two-stage recursive model index).

TEST INFRASTRUCTURE ONLY: the tests, smoke() and the benchmark's CPU leg may
import this module; the join library never does, and nothing here is shared
with the CUDA path.

The model approximates the empirical CDF of a sorted key sample, the role the
paper gives to its equi-height CDF of the runs (Sec. 4.1-4.2, Fig. 8): a key's
predicted CDF value times a run's length predicts where the key's merge starts
in that run (Sec. 3.2.2), and times P predicts its partition (Sec. 4.3).  The
model's output is only ever a starting point for an exact search, so it never
changes a join result.

Stage 1 (the root) is a multilayer perceptron over the normalised key
x = (key - kmin) / (kmax - kmin):

    h1 = relu(W1 x + b1)          W1, b1 in R^32
    h2 = relu(W2 h1 + b2)         W2 in R^{32x32} (row j = output j), b2 in R^32
    yhat = W3 . h2 + b3           W3 in R^32, b3 in R

trained by full-batch Adam (Kingma & Ba 2015) on the mean squared error
against the sample's rank fractions.  Stage 2 holds L linear leaves; the root
picks leaf floor(L * yhat) (clamped), and each leaf is the least-squares line
of the rank fraction on the key's exact integer offset from the leaf's smallest
training key.

Parameter vector layout (1153 values): W1[32], b1[32], W2[32*32], b2[32], W3[32], b3[1].
"""
import numpy as np

H = 32
NPARAM = H + H + H * H + H + H + 1
O_W1, O_B1, O_W2, O_B2, O_W3, O_B3 = 0, H, 2 * H, 2 * H + H * H, 3 * H + H * H, 4 * H + H * H


def unpack(theta):
    t = np.asarray(theta, dtype=np.float64)
    assert t.shape == (NPARAM,)
    return (t[O_W1:O_B1], t[O_B1:O_W2], t[O_W2:O_B2].reshape(H, H), t[O_B2:O_W3], t[O_W3:O_B3], t[O_B3])


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([W1, b1, np.asarray(W2).reshape(-1), b2, W3, [b3]]).astype(np.float64)


def initial_theta():
    """Deterministic start: hinge features relu(x - j/32) passed through an identity
    middle layer and read out by the first one, i.e. the model starts as yhat = x
    (the CDF of uniformly spread keys)."""
    W1 = np.ones(H)
    b1 = -np.arange(H) / H
    W2 = np.eye(H)
    b2 = np.zeros(H)
    W3 = np.zeros(H)
    W3[0] = 1.0
    return pack(W1, b1, W2, b2, W3, 0.0)


def forward(theta, x):
    """Root output yhat for a vector of normalised keys x (FP64)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    x = np.asarray(x, dtype=np.float64)
    a1 = np.outer(x, W1) + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    return h2 @ W3 + b3


def loss_grad(theta, x, y):
    """Mean squared error over the batch and its gradient, by the chain rule written out layer by layer.

    The ReLU derivative is taken as 1 where its input is > 0 and 0 elsewhere."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = x.shape[0]
    a1 = np.outer(x, W1) + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    yhat = h2 @ W3 + b3
    r = yhat - y
    loss = float(np.mean(r * r))
    g = 2.0 * r / n                       # dL/dyhat per sample
    dW3 = h2.T @ g
    db3 = g.sum()
    da2 = np.outer(g, W3) * (a2 > 0)      # dL/da2
    dW2 = da2.T @ h1                      # [j, k] = sum_i da2[i, j] h1[i, k]
    db2 = da2.sum(axis=0)
    da1 = (da2 @ W2) * (a1 > 0)           # dL/da1
    dW1 = da1.T @ x
    db1 = da1.sum(axis=0)
    return loss, pack(dW1, db1, dW2, db2, dW3, db3)


def adam_step(theta, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1) with bias-corrected moments; returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def train(theta, x, y, steps, lr):
    """Full-batch Adam from theta for `steps` steps; returns (theta, loss history before each step)."""
    m = np.zeros(NPARAM)
    v = np.zeros(NPARAM)
    hist = []
    for t in range(1, steps + 1):
        loss, g = loss_grad(theta, x, y)
        hist.append(loss)
        theta, m, v = adam_step(theta, m, v, g, t, lr)
    return theta, hist


def leaf_of(yhat, nleaf):
    """Leaf picked by the root: floor(nleaf * yhat) clamped to [0, nleaf)."""
    return np.clip(np.floor(np.asarray(yhat, dtype=np.float64) * nleaf), 0, nleaf - 1).astype(np.int64)


def fit_leaves(keys, y, leaf, nleaf):
    """Per-leaf least squares of y on d = key - base (base = the leaf's smallest key).

    Slope = sum((d - mean d)(y - mean y)) / sum((d - mean d)^2), intercept = mean y -
    slope * mean d (centred sums, so huge key offsets lose no precision).  Returns
    (base u64[nleaf], slope f64[nleaf], intercept f64[nleaf], count i64[nleaf]).  A
    leaf whose keys are all equal gets slope 0 and the mean of its y; an empty leaf
    gets base 0, slope 0 and intercept (l + 0.5) / nleaf (the root's own estimate)."""
    keys = np.asarray(keys, dtype=np.uint64)
    y = np.asarray(y, dtype=np.float64)
    leaf = np.asarray(leaf, dtype=np.int64)
    base = np.zeros(nleaf, dtype=np.uint64)
    a = np.zeros(nleaf)
    b = (np.arange(nleaf) + 0.5) / nleaf
    cnt = np.bincount(leaf, minlength=nleaf)
    for l in np.nonzero(cnt)[0]:
        sel = leaf == l
        k = keys[sel]
        base[l] = k.min()
        d = (k - base[l]).astype(np.float64)
        yy = y[sel]
        dm, ym = d.mean(), yy.mean()
        sxx = ((d - dm) ** 2).sum()
        if sxx > 0:
            a[l] = ((d - dm) * (yy - ym)).sum() / sxx
            b[l] = ym - a[l] * dm
        else:
            a[l] = 0.0
            b[l] = ym
    return base, a, b, cnt


def leaf_predict(keys, leaf, base, a, b):
    """Stage-2 prediction a[l] * (key - base[l]) + b[l] with the signed exact offset."""
    keys = np.asarray(keys, dtype=np.uint64)
    bl = base[leaf]
    d = np.where(keys >= bl, (keys - bl).astype(np.float64), -((bl - keys).astype(np.float64)))
    return a[leaf] * d + b[leaf]
