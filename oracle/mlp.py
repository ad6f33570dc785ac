"""Oracle of the tolerance controller's network: TEST INFRASTRUCTURE ONLY.

The controller is not in the paper. Its network is a plain multilayer perceptron
x -> tanh(W1 x + b1) -> tanh(W2 h1 + b2) -> W3 h2 + b3 (one output: the predicted log10
of a product's relative error), trained on the mean squared error
L = (1 / 2N) sum_n (y_hat_n - y_n)^2 with Adam (Kingma and Ba, "Adam: A Method for
Stochastic Optimization", ICLR 2015: m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
theta <- theta - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)).
Everything here is FP64 numpy. Parameters are one flat vector in the order
W1 (H x F, row-major), b1 (H), W2 (H x H), b2 (H), W3 (1 x H), b3 (1).
"""
from __future__ import annotations

import numpy as np


def sizes(F: int, H: int) -> list[tuple[int, ...]]:
    return [(H, F), (H,), (H, H), (H,), (1, H), (1,)]


def unpack(theta: np.ndarray, F: int, H: int) -> list[np.ndarray]:
    out, o = [], 0
    for s in sizes(F, H):
        k = int(np.prod(s))
        out.append(theta[o:o + k].reshape(s))
        o += k
    assert o == theta.size
    return out


def n_params(F: int, H: int) -> int:
    return sum(int(np.prod(s)) for s in sizes(F, H))


def forward(theta, X, F, H):
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, dtype=np.float64), F, H)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return (h2 @ W3.T + b3)[:, 0], (h1, h2)


def loss_and_grad(theta, X, y, F, H):
    """Loss and its exact gradient (back-propagation written out)."""
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, dtype=np.float64), F, H)
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    N = X.shape[0]
    yh, (h1, h2) = forward(theta, X, F, H)
    r = yh - y
    L = 0.5 * np.mean(r * r)
    d3 = r[:, None] / N                     # dL/d yhat
    gW3 = d3.T @ h2
    gb3 = d3.sum(0)
    d2 = (d3 @ W3) * (1.0 - h2 * h2)
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (1.0 - h1 * h1)
    gW1 = d1.T @ X
    gb1 = d1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, g


def grad_abs_terms(theta, X, y, F, H):
    """Sum over samples of |per-sample gradient term|, the scale of the rounding error
    of a per-component sum over N samples."""
    X = np.asarray(X, dtype=np.float64)
    tot = np.zeros(n_params(F, H))
    for n in range(X.shape[0]):
        _, g = loss_and_grad(theta, X[n:n + 1], np.asarray(y)[n:n + 1], F, H)
        tot += np.abs(g) / X.shape[0]
    return tot


class Adam:
    def __init__(self, theta, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.theta = np.array(theta, dtype=np.float64)
        self.m = np.zeros_like(self.theta)
        self.v = np.zeros_like(self.theta)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        self.theta = self.theta - self.lr * mh / (np.sqrt(vh) + self.eps)
        return self.theta


# ---- features of a product (the controller's input) ----
HIST = 16
N_FEATURES = 4 * HIST + 5
# squared-norm thresholds of the decade bins: 10^-2, 10^-4, ..., 10^-30
_DECADE2 = [float(f"1e-{2 * (q + 1)}") for q in range(HIST - 1)]


def tier_hist(norm2: np.ndarray) -> tuple[np.ndarray, int]:
    """16-bin histogram of one tier's blocks by decades of norm below the tier's largest
    norm, as float32 fractions of its nonzero blocks; and the nonzero count. A block goes
    to bin q when max^2 * 10^-2(q+1) <= norm^2 < max^2 * 10^-2q (bin 15 collects the
    rest), the comparison taken in FP64."""
    v = np.asarray(norm2, dtype=np.float64).ravel()
    m = float(v.max()) if v.size else 0.0
    thr = [m * c for c in _DECADE2]
    counts = np.zeros(HIST, dtype=np.int64)
    nz = 0
    for x in v:
        if not x > 0.0:
            continue
        nz += 1
        b = 0
        while b < HIST - 1 and x < thr[b]:
            b += 1
        counts[b] += 1
    frac = np.array([np.float32(c) / np.float32(nz) if nz else np.float32(0.0) for c in counts],
                    dtype=np.float32)
    return frac, nz


def tree_features(tree, nb: int) -> np.ndarray:
    """Per-operand part: leaf-tier and next-tier histograms, fraction of nonzero leaves,
    log10 of the Frobenius norm (from the root of the norm tree)."""
    k = tree.kmax
    hl, nzl = tier_hist(tree.norm2(k))
    hp, _ = tier_hist(tree.norm2(max(k - 1, 0)))
    root = float(tree.norm2(0).ravel()[0])
    out = np.zeros(2 * HIST + 2, dtype=np.float32)
    out[:HIST], out[HIST:2 * HIST] = hl, hp
    out[2 * HIST] = np.float32(nzl) / np.float32(nb * nb)
    out[2 * HIST + 1] = np.float32(0.5 * np.log10(root)) if root > 0 else np.float32(-300.0)
    return out


def flat_bound32(treeA, treeB, taus) -> np.ndarray:
    """Flat leaf bound at each tau: the sum of p = ||A_ik|| ||B_kj|| over leaf triples
    with p < tau, with the leaf norms, p and the comparison in FP32 (tau rounded to
    FP32), the sum in FP64. A plain triple loop over (i, k) and a vector over j."""
    nA = np.sqrt(treeA.norm2(treeA.kmax)).astype(np.float32)
    nB = np.sqrt(treeB.norm2(treeB.kmax)).astype(np.float32)
    thr = np.asarray(taus, dtype=np.float64).astype(np.float32)
    out = np.zeros(thr.size)
    NB = nA.shape[0]
    for i in range(NB):
        for k in range(NB):
            if nA[i, k] == 0:
                continue
            p = nA[i, k] * nB[k, :]                 # FP32 products
            p = p[p > 0]
            for q, t in enumerate(thr):
                out[q] += float(np.sum(p[p < t].astype(np.float64)))
    return out


def features(treeA, nbA: int, treeB, nbB: int, tau: float, bound: float | None = None) -> np.ndarray:
    """The network's input for the product A B at tolerance tau (the flat bound at tau
    is computed unless given)."""
    fa, fb = tree_features(treeA, nbA), tree_features(treeB, nbB)
    la, lb = float(fa[2 * HIST + 1]), float(fb[2 * HIST + 1])
    if bound is None:
        bound = flat_bound32(treeA, treeB, [tau])[0]
    f = np.zeros(N_FEATURES, dtype=np.float32)
    f[:2 * HIST], f[2 * HIST:4 * HIST] = fa[:2 * HIST], fb[:2 * HIST]
    f[4 * HIST] = np.float32((np.log10(tau) - la - lb) / 8.0)
    f[4 * HIST + 1] = np.float32((la + lb) / 8.0)
    f[4 * HIST + 2], f[4 * HIST + 3] = fa[2 * HIST], fb[2 * HIST]
    lr = (np.log10(bound) - la - lb) / 8.0 if bound > 0 else -2.0
    f[4 * HIST + 4] = np.float32(max(lr, -2.0))
    return f


def near_threshold(norm2: np.ndarray, rel: float = 1e-12) -> int:
    """Blocks whose squared norm lies within `rel` of a bin threshold: the only ones whose
    bin may differ between two norm trees equal to rounding."""
    v = np.asarray(norm2, dtype=np.float64).ravel()
    m = float(v.max()) if v.size else 0.0
    thr = np.array([m * c for c in _DECADE2])
    if m == 0.0:
        return 0
    close = np.abs(v[:, None] - thr[None, :]) <= rel * thr[None, :]
    return int(close.any(axis=1).sum())
