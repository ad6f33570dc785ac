"""GPU parity of the tolerance controller: its network kernels (forward, backward, Adam)
against the FP64 oracle in oracle/mlp.py, its features against the oracle's features
of the same matrices, and its tolerance choice against the oracle's network.

Tolerances (FP32 kernels against an FP64 oracle):
  forward   |y_gpu - y| <= 2^-16 (1 + |y|): each pre-activation is a sum of at most
            F + 1 = 69 FP32 products (error <= 69 u of the absolute sum), two tanh layers
            and the output sum add about 2H u, so |err| ~ (F + 3H) u ~ 2^-17 of the
            absolute values, which are O(1) here; a factor two of margin.
  gradient  |g_gpu - g| <= 2^-15 T_q + 1e-7 max|g|, T_q = sum over samples of the
            absolute per-sample terms of component q: the per-sample chain adds about
            2^-17 relative, the sum over N <= 256 samples N u <= 2^-16.
  Adam      fed the same FP32 gradients, the trajectories differ only by the FP32
            rounding of the update: per step <= 4 u |theta| + 10 u lr, so after t
            steps |dtheta| <= t 2^-24 (4 max|theta| + 10 lr) (sum of per-step bounds).
"""
import numpy as np
import pytest

import oracle
from oracle import mlp as M
from paper_1011_3534_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

F, H = 69, 32
U = 2.0 ** -24


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1011_3534_gb300 import spamm
    return spamm


@pytest.fixture(scope="module")
def ctx(S):
    c = S.spamm_ctx_create(0, torch.cuda.current_stream())
    yield c
    S.spamm_ctx_destroy(c)


def data(N, seed):
    r = np.random.default_rng(seed)
    X = r.normal(0, 1, (N, F)).astype(np.float32)
    y = r.normal(0, 1, N).astype(np.float32)
    return X, y


def test_forward_matches_oracle(S, ctx):
    m = S.Mlp(ctx, F, H, seed=11)
    th = m.get_params()
    assert th.size == M.n_params(F, H)
    X, _ = data(300, 1)               # 300 samples: more than two 128-thread blocks
    got = m.forward(X)
    ref, _ = M.forward(th.astype(np.float64), X.astype(np.float64), F, H)
    assert np.all(np.abs(got - ref) <= 2.0 ** -16 * (1 + np.abs(ref)))
    m.free()


def test_initialisation_is_the_stated_uniform(S, ctx):
    m = S.Mlp(ctx, F, H, seed=3)
    W1, b1, W2, b2, W3, b3 = M.unpack(m.get_params().astype(np.float64), F, H)
    assert np.all(b1 == 0) and np.all(b2 == 0) and np.all(b3 == 0)
    assert np.abs(W1).max() <= 1 / np.sqrt(F) and np.abs(W2).max() <= 1 / np.sqrt(H)
    assert np.abs(W1).max() > 0.9 / np.sqrt(F)            # the whole interval is used
    m2 = S.Mlp(ctx, F, H, seed=3)
    assert np.array_equal(m.get_params(), m2.get_params())  # reproducible from the seed
    m.free()
    m2.free()


@pytest.mark.parametrize("N", [1, 37, 256])
def test_gradient_matches_oracle(S, ctx, N):
    m = S.Mlp(ctx, F, H, seed=5)
    th = m.get_params().astype(np.float64)
    X, y = data(N, 2 + N)
    L, g = m.gradient(X, y)
    Lr, gr = M.loss_and_grad(th, X, y, F, H)
    T = M.grad_abs_terms(th, X, y, F, H)
    tol = 2.0 ** -15 * T + 1e-7 * np.abs(gr).max()
    bad = np.abs(g - gr) > tol
    assert not bad.any(), (np.argwhere(bad)[:5], g[bad][:5], gr[bad][:5])
    assert abs(L - Lr) <= 2.0 ** -15 * (Lr + 1e-30)
    m.free()


def test_gradient_matches_finite_differences_of_the_gpu_loss(S, ctx):
    # central differences of the GPU's own FP32 loss, on the largest components: the
    # step h = 1e-2 keeps the FP32 rounding of the loss (~u L / h) below 1e-4 L
    m = S.Mlp(ctx, F, H, seed=8)
    th = m.get_params()
    X, y = data(64, 9)
    _, g = m.gradient(X, y)
    idx = np.argsort(-np.abs(g))[:12]
    h = 1e-2
    for q in idx:
        tp, tm = th.copy(), th.copy()
        tp[q] += h
        tm[q] -= h
        m.set_params(tp)
        Lp, _ = m.gradient(X, y)
        m.set_params(tm)
        Lm, _ = m.gradient(X, y)
        num = (Lp - Lm) / (2 * h)
        assert abs(num - g[q]) <= 2e-2 * abs(g[q]) + 1e-5, (q, num, g[q])
    m.free()


def test_adam_matches_oracle_for_100_steps(S, ctx):
    m = S.Mlp(ctx, F, H, seed=6)
    th0 = m.get_params().astype(np.float64)
    ad = M.Adam(th0, lr=1e-3)
    X, y = data(128, 12)
    r = np.random.default_rng(13)
    worst = np.abs(th0).max()
    for t in range(1, 101):
        # the gradient at the GPU's parameters, from the oracle, in FP32
        cur = m.get_params().astype(np.float64)
        g = M.loss_and_grad(cur, X, y, F, H)[1].astype(np.float32)
        g += r.normal(0, 1e-3, g.size).astype(np.float32) * (t % 7 == 0)   # some noisy steps
        m.adam_apply(g, 1e-3)
        ad.step(g.astype(np.float64))
        worst = max(worst, np.abs(ad.theta).max())
        tol = t * U * (4 * worst + 10 * 1e-3)
        d = np.abs(m.get_params().astype(np.float64) - ad.theta).max()
        assert d <= tol, (t, d, tol)
    m.free()


def test_adam_step_end_to_end_follows_oracle(S, ctx):
    # the library's own gradients inside the step: 50 full-batch steps stay close to the
    # FP64 trajectory (gradient and update rounding both enter; a wrong sign, beta or
    # bias correction moves theta by about lr per step)
    m = S.Mlp(ctx, F, H, seed=4)
    ad = M.Adam(m.get_params().astype(np.float64), lr=1e-3)
    X, y = data(96, 21)
    for _ in range(50):
        m.adam_step(X, y, 1e-3)
        ad.step(M.loss_and_grad(ad.theta, X, y, F, H)[1])
    d = np.abs(m.get_params().astype(np.float64) - ad.theta)
    assert np.median(d) < 1e-3 * 1e-3 * 50 and d.max() < 0.5 * 1e-3 * 50
    m.free()


def test_training_reduces_loss(S, ctx):
    m = S.Mlp(ctx, 3, 16, seed=1)
    r = np.random.default_rng(1)
    X = r.uniform(-1, 1, (2000, 3)).astype(np.float32)
    y = np.sin(X @ np.array([1.0, -2.0, 0.5])).astype(np.float32)
    L0, _ = m.gradient(X, y)
    L = m.train(X, y, epochs=40, batch=64, lr=3e-3, seed=2)
    assert L < 0.05 * L0
    # the reported loss is the oracle's loss at the trained parameters
    Lr, _ = M.loss_and_grad(m.get_params().astype(np.float64), X, y, 3, 16)
    assert abs(L - Lr) <= 1e-5 * Lr + 1e-9
    m.free()


def _tree(S, ctx, A, leaf, flags):
    return S.spamm_tree_build(ctx, torch.from_numpy(A).cuda(), A.shape[0], leaf, flags)


@pytest.mark.parametrize("n,leaf,kind", [(1000, 64, "alg"), (1536, 32, "exp"), (40, 64, "exp"), (4096, 64, "alg")])
def test_features_match_oracle(S, ctx, n, leaf, kind):
    A = W.algebraic_decay(n, 2, 0) if kind == "alg" else W.exp_decay(n, 0.85, 1, 0)
    B = W.exp_decay(n, 0.9, 1, 1)
    tA = _tree(S, ctx, A, leaf, S.SPAMM_KEEP_FP64)
    tB = _tree(S, ctx, B, leaf, S.SPAMM_KEEP_FP64)
    TA, TB = oracle.Tree(A, leaf), oracle.Tree(B, leaf)
    nb = -(-n // leaf)
    for tau in (1e-10, 1e-6, 3e-3):
        got = S.spamm_features(tA, tB, tau)
        ref = M.features(TA, nb, TB, nb, tau)
        # histograms: integer work, exact but for blocks within rounding of a threshold
        slack = []
        for T in (TA, TB):
            k = T.kmax
            slack += [M.near_threshold(T.norm2(k)), M.near_threshold(T.norm2(max(k - 1, 0)))]
        for part, s in zip(range(4), slack):
            a, b = got[16 * part:16 * (part + 1)], ref[16 * part:16 * (part + 1)]
            if s == 0:
                assert np.array_equal(a, b), (part, a, b)
            else:
                assert np.abs(a - b).sum() <= 2 * s / max(1, (b > 0).sum()), (part, a, b)
        assert got[66] == ref[66] and got[67] == ref[67]
        np.testing.assert_allclose(got[64:66], ref[64:66], rtol=1e-6, atol=1e-6)
        # flat bound: the same FP32 decisions; FP32 partial sums (about NB terms per
        # thread) against the oracle's FP64 sum: 1e-5 relative, i.e. 1e-5 / (8 ln 10)
        # in the scaled log10 feature
        assert abs(got[68] - ref[68]) <= 1e-6, (got[68], ref[68])
    S.spamm_tree_free(tA)
    S.spamm_tree_free(tB)


def test_tau_select_matches_oracle_network(S, ctx):
    n, leaf = 2048, 64
    A = W.algebraic_decay(n, 2, 0)
    tA = _tree(S, ctx, A, leaf, S.SPAMM_KEEP_FP64 | S.SPAMM_SYMMETRIC)
    TA = oracle.Tree(A, leaf)
    nb = n // leaf
    m = S.Mlp(ctx, F, H, seed=17)
    th = m.get_params().astype(np.float64)
    lo, hi, G = 1e-12, 1e-2, 37
    grid = np.log10(lo) + np.arange(G) * (np.log10(hi) - np.log10(lo)) / (G - 1)
    bounds = M.flat_bound32(TA, TA, 10.0 ** grid)
    feats = np.stack([M.features(TA, nb, TA, nb, 10.0 ** g, bound=b) for g, b in zip(grid, bounds)])
    pred, _ = M.forward(th, feats.astype(np.float64), F, H)
    for q in (3, 12, 20, 30):
        budget = 10.0 ** float(pred[q])     # a budget met by some grid points, not all
        tau = S.spamm_tau_select(m, tA, tA, budget, lo, hi)
        ok = np.nonzero(pred <= np.log10(budget))[0]
        want = ok.max() if ok.size else 0
        g = int(round((np.log10(tau) - grid[0]) / (grid[1] - grid[0])))
        assert abs(np.log10(tau) - grid[g]) < 1e-9
        if g != want:   # only predictions within FP32 rounding of the budget may flip
            assert np.abs(pred[[g, want]] - np.log10(budget)).min() < 1e-4, (g, want)
    # a constant network: all or nothing
    z = np.zeros(m.P, dtype=np.float32)
    z[-1] = -5.0
    m.set_params(z)
    assert abs(S.spamm_tau_select(m, tA, tA, 1e-4, lo, hi) / hi - 1) < 1e-12
    assert abs(S.spamm_tau_select(m, tA, tA, 1e-6, lo, hi) / lo - 1) < 1e-12
    m.free()
    S.spamm_tree_free(tA)


def test_tree_distance(S, ctx):
    n, leaf = 900, 32
    A = W.algebraic_decay(n, 2, 0)
    B = A + 1e-3 * W.exp_decay(n, 0.8, 1, 3)
    tA = _tree(S, ctx, A, leaf, S.SPAMM_KEEP_FP64)
    tB = _tree(S, ctx, B, leaf, S.SPAMM_KEEP_FP64)
    d, r = S.spamm_tree_distance(tA, tB)
    assert abs(d - np.linalg.norm(A - B)) <= 1e-12 * np.linalg.norm(A - B)
    assert abs(r - np.linalg.norm(B)) <= 1e-12 * np.linalg.norm(B)
    S.spamm_tree_free(tA)
    S.spamm_tree_free(tB)
