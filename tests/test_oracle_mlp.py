"""Pins of the MLP oracle (CPU): gradients against central finite differences, a
hand-worked tiny network, and Adam against its closed form on a quadratic."""
import numpy as np

from oracle import mlp as M


def test_gradient_matches_finite_differences():
    F, H = 5, 4
    r = np.random.default_rng(0)
    theta = r.normal(0, 0.5, M.n_params(F, H))
    X, y = r.normal(size=(7, F)), r.normal(size=7)
    L, g = M.loss_and_grad(theta, X, y, F, H)
    h = 1e-6
    for i in range(theta.size):
        e = np.zeros_like(theta)
        e[i] = h
        num = (M.loss_and_grad(theta + e, X, y, F, H)[0] - M.loss_and_grad(theta - e, X, y, F, H)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, num, g[i])


def test_hand_worked_single_unit():
    # F = H = 1, all weights 1, biases 0: h1 = tanh(x), h2 = tanh(tanh(x)), yhat = h2
    F, H = 1, 1
    theta = np.array([1.0, 0.0, 1.0, 0.0, 1.0, 0.0])
    yh, _ = M.forward(theta, np.array([[0.5]]), F, H)
    assert abs(yh[0] - np.tanh(np.tanh(0.5))) < 1e-15
    L, g = M.loss_and_grad(theta, np.array([[0.5]]), np.array([0.0]), F, H)
    h1, h2 = np.tanh(0.5), np.tanh(np.tanh(0.5))
    assert abs(L - 0.5 * h2 * h2) < 1e-15
    assert abs(g[4] - h2 * h2) < 1e-15 and abs(g[5] - h2) < 1e-15          # dW3, db3
    d2 = h2 * (1 - h2 * h2)
    assert abs(g[2] - d2 * h1) < 1e-15                                     # dW2
    assert abs(g[0] - d2 * (1 - h1 * h1) * 0.5) < 1e-15                    # dW1


def test_adam_first_step_and_convergence():
    # first Adam step: bias-corrected m = g and v = g^2, so theta moves by -lr g / (|g| + eps)
    a = M.Adam(np.zeros(3), lr=0.1)
    g = np.array([2.0, -0.5, 1e-3])
    th = a.step(g)
    np.testing.assert_allclose(th, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # on f(x) = |x - c|^2 / 2 Adam converges to c
    c = np.array([1.0, -2.0, 3.0])
    a = M.Adam(np.zeros(3), lr=0.05)
    for _ in range(3000):
        a.step(a.theta - c)
    np.testing.assert_allclose(a.theta, c, atol=1e-3)


def test_training_reduces_loss():
    F, H = 3, 8
    r = np.random.default_rng(1)
    X = r.uniform(-1, 1, (256, F))
    y = np.sin(X @ np.array([1.0, -2.0, 0.5]))
    theta = r.normal(0, 0.5, M.n_params(F, H))
    L0 = M.loss_and_grad(theta, X, y, F, H)[0]
    a = M.Adam(theta, lr=1e-2)
    for _ in range(500):
        a.step(M.loss_and_grad(a.theta, X, y, F, H)[1])
    assert M.loss_and_grad(a.theta, X, y, F, H)[0] < 0.1 * L0


def _block_diag(norms, b):
    """Block-diagonal matrix whose diagonal leaf i is filled with one value, so its
    Frobenius norm is norms[i]."""
    nbk = len(norms)
    A = np.zeros((nbk * b, nbk * b))
    for i, v in enumerate(norms):
        A[i * b:(i + 1) * b, i * b:(i + 1) * b] = v / b
    return A


def test_features_of_a_constructed_matrix():
    import oracle
    b = 16
    norms = [1.0, 10 ** -0.5, 10 ** -1.5, 10 ** -2.5, 10 ** -3.5, 10 ** -5.5, 1e-17, 0.5]
    A = _block_diag(norms, b)
    T = oracle.Tree(A, b)
    f = M.tree_features(T, 8)
    leaf = np.zeros(16)
    leaf[[0, 1, 2, 3, 5, 15]] = [3, 1, 1, 1, 1, 1]
    np.testing.assert_array_equal(f[:16], (leaf / 8).astype(np.float32))
    # the tier above: diagonal parents hold leaves (0,1), (2,3), (4,5), (6,7); their
    # norms relative to the largest, sqrt(1.1), are 1, 0.0303, 3.0e-4 and 0.477
    par = np.zeros(16)
    par[[0, 1, 3]] = [2, 1, 1]
    np.testing.assert_array_equal(f[16:32], (par / 4).astype(np.float32))
    assert f[32] == np.float32(8 / 64)
    tot2 = 1.0 + 0.1 + 10 ** -3 + 10 ** -5 + 10 ** -7 + 10 ** -11 + 1e-34 + 0.25
    assert abs(f[33] - 0.5 * np.log10(tot2)) < 1e-6
    # the product features put A's part first, B's second, then the scaled logs
    g = M.features(T, 8, T, 8, 1e-8)
    np.testing.assert_array_equal(g[:32], f[:32])
    np.testing.assert_array_equal(g[32:64], f[:32])
    assert abs(g[64] - (-8 - np.log10(tot2)) / 8) < 1e-6
    assert abs(g[65] - np.log10(tot2) / 8) < 1e-6
    assert g[66] == g[67] == np.float32(0.125)
    # flat bound: A is block diagonal, so the only leaf products are (i, i, i) with
    # p = norm_i^2; below 1e-8 lie 1e-11 and 1e-34
    assert abs(g[68] - (np.log10(1e-11 + 1e-34) - np.log10(tot2)) / 8) < 1e-6
    b = M.flat_bound32(T, T, [1e-8, 2e-3, 1e-40])
    np.testing.assert_allclose(b, [1e-11 + 1e-34, 1e-3 + 1e-5 + 1e-7 + 1e-11 + 1e-34, 0.0], rtol=1e-6)
    assert M.features(T, 8, T, 8, 1e-40)[68] == np.float32(-2.0)     # nothing below tau: the floor


def test_flat_bound32_matches_the_fp64_oracle_bound():
    # the FP32 bound against the C oracle's FP64 flat bound (an independent loop) on a
    # random decaying matrix, away from ties at the thresholds
    import oracle
    n = 300
    r = np.random.default_rng(3)
    d = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :])
    A = r.uniform(-1, 1, (n, n)) * 0.8 ** d
    T = oracle.Tree(A, 16)
    for tau in (1e-9, 1e-5, 1e-2):
        got = M.flat_bound32(T, T, [tau])[0]
        ref = oracle.flat_bound(T, T, tau)
        assert abs(got - ref) <= 1e-5 * ref + 1e-300, (tau, got, ref)


def test_feature_bins_follow_the_decades():
    # a block exactly one decade down is at the bottom of bin 0; a hair below, in bin 1
    frac, nz = M.tier_hist(np.array([1.0, 1e-2, 1e-2 * (1 - 1e-9), 0.0]))
    assert nz == 3
    assert frac[0] == np.float32(2 / 3) and frac[1] == np.float32(1 / 3)
    assert M.near_threshold(np.array([1.0, 1e-2, 0.5])) == 1
