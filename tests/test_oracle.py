"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed form, a
hand-worked case, numpy's own routines, brute force, or a bound. The mutant test at
the end plants known mistakes in copies of the oracle and checks that some pin fails.
"""
import numpy as np
import pytest

import oracle
from paper_1011_3534_gb300 import workloads as W

EPS = np.finfo(np.float64).eps


def blocks_norm2_numpy(A, b):
    """Squared Frobenius norm of each b x b block of the zero-padded A (numpy)."""
    n = A.shape[0]
    nb = -(-n // b)
    NB = 1
    while NB < nb:
        NB *= 2
    P = np.zeros((NB * b, NB * b))
    P[:n, :n] = A
    return (P.reshape(NB, b, NB, b) ** 2).sum(axis=(1, 3)), P, NB


def brute_triples_numpy(nA2, nB2, tau):
    """All (i, j, k) with sqrt(nA2[i,k]) * sqrt(nB2[k,j]) >= tau, lexicographic."""
    p = np.sqrt(nA2)[:, None, :] * np.sqrt(nB2).T[None, :, :]  # [i, j, k]
    i, j, k = np.nonzero(~(p < tau))
    return np.stack([i, j, k], axis=1).astype(np.uint32)


DEPTH_TAU = 3e-2   # the depth-scaled pin's tau (no tier product within 1e-6 of its threshold)


def tier_norm2_numpy(nL2, l, kmax):
    """Squared norms of tier l from the leaf tier, by summing 2^s x 2^s groups (numpy)."""
    s = 1 << (kmax - l)
    d = nL2.shape[0] // s
    return nL2.reshape(d, s, d, s).sum(axis=(1, 3))


def brute_depth_triples_numpy(A, B, b, tau, margin=None):
    """Leaf triples (i, j, k) of the depth-scaled recursion, lexicographic: every ancestor
    (i, j, k) >> s at tier l = kmax - s has ||A^l|| ||B^l|| >= tau * 8^-l. With `margin`,
    also the smallest relative distance of a tested product from its threshold."""
    nA2, _, NB = blocks_norm2_numpy(A, b)
    nB2, _, _ = blocks_norm2_numpy(B, b)
    kmax = NB.bit_length() - 1
    alive = np.ones((1, 1, 1), dtype=bool)
    gap = np.inf
    for l in range(kmax + 1):
        a2, b2 = tier_norm2_numpy(nA2, l, kmax), tier_norm2_numpy(nB2, l, kmax)
        p = np.sqrt(a2)[:, None, :] * np.sqrt(b2).T[None, :, :]     # [i, j, k] at tier l
        tl = tau * 8.0 ** -l
        parent = alive.repeat(2, 0).repeat(2, 1).repeat(2, 2) if l else alive
        if parent.any():
            gap = min(gap, float(np.min(np.abs(p[parent] - tl)) / tl))
        alive = parent & ~(p < tl)
    i, j, k = np.nonzero(alive)
    out = np.stack([i, j, k], axis=1).astype(np.uint32)
    return (out, gap) if margin else out


def spamm_numpy_from_triples(P_A, P_B, trip, b, n):
    NB = P_A.shape[0] // b
    C = np.zeros_like(P_A)
    for i, j, k in trip:
        C[i * b:(i + 1) * b, j * b:(j + 1) * b] += (
            P_A[i * b:(i + 1) * b, k * b:(k + 1) * b] @ P_B[k * b:(k + 1) * b, j * b:(j + 1) * b])
    return C[:n, :n]


def rng_matrix(n, seed, sym=False, decay=0.8):
    r = np.random.default_rng(seed)
    d = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :])
    M = r.uniform(-1, 1, (n, n)) * decay ** d
    return (M + M.T) / 2 if sym else M


# ---------------------------------------------------------------- norm pyramid (Eq. 1)

def test_norms_constant_closed_form():
    # ||c * 1_{b x b}||_F^2 = c^2 b^2 exactly; a tier-l block covers 4^(kmax-l) leaves
    n, b, c = 64, 8, 2.0
    T = oracle.Tree(np.full((n, n), c), b)
    assert T.kmax == 3
    for l in range(T.kmax + 1):
        expect = c * c * b * b * 4 ** (T.kmax - l)
        assert np.all(T.norm2(l) == expect)


def test_norms_padded_constant():
    # n = 40, b = 16: nb = 3, NB = 4; block (2, 2) holds an 8 x 8 corner of ones
    T = oracle.Tree(np.ones((40, 40)), 16)
    leaf = T.norm2(2)
    assert T.NB == 4
    assert leaf[0, 0] == 256 and leaf[0, 2] == 128 and leaf[2, 2] == 64
    assert np.all(leaf[3, :] == 0) and np.all(leaf[:, 3] == 0)
    assert T.norm2(0)[0, 0] == 1600.0


@pytest.mark.parametrize("n,b", [(96, 16), (100, 8), (1, 4), (33, 32)])
def test_norms_vs_numpy(n, b):
    A = rng_matrix(n, 1)
    T = oracle.Tree(A, b)
    ref, _, NB = blocks_norm2_numpy(A, b)
    assert T.NB == NB
    np.testing.assert_allclose(T.norm2(T.kmax), ref, rtol=1e-13, atol=0)
    root = np.linalg.norm(A) ** 2
    assert abs(T.norm2(0)[0, 0] - root) <= 1e-13 * root


def test_norms_monotone_bitwise():
    T = oracle.Tree(W.algebraic_decay(256, 2, 0), 16)
    for l in range(T.kmax):
        par, ch = T.norm2(l), T.norm2(l + 1)
        for a in range(2):
            for c in range(2):
                assert np.all(par >= ch[a::2, c::2])


# ---------------------------------------------------------------- triples (Eq. 4)

def test_hand_worked_2x2():
    # b = 1, A = B = [[1, .01], [.01, 1]], tau = 1e-3: leaf products |A_ik||B_kj| are
    # 1 for (0,0,0), (1,1,1); .01 for (0,1,0), (0,1,1), (1,0,0), (1,0,1); 1e-4 for
    # (0,0,1), (1,1,0), which are dropped. C~ = [[1, .02], [.02, 1]].
    A = np.array([[1.0, 0.01], [0.01, 1.0]])
    T = oracle.Tree(A, 1)
    r = oracle.spamm(T, T, 1e-3, triples=True, stats=True)
    got = {tuple(int(x) for x in t) for t in r["triples"]}
    assert got == {(0, 0, 0), (1, 1, 1), (0, 1, 0), (0, 1, 1), (1, 0, 0), (1, 0, 1)}
    assert np.array_equal(r["C"], np.array([[1.0, 0.02], [0.02, 1.0]]))
    st = r["stats"]
    assert st.tested == [1, 8] and st.culled == [0, 2] and st.leaf_products == 6
    assert abs(st.culled_bound[1] - 2e-4) < 1e-18


@pytest.mark.parametrize("n,b,tau,sym", [(128, 16, 1e-3, True), (200, 16, 1e-4, False),
                                         (256, 32, 1e-6, False), (64, 4, 1e-2, False)])
def test_recursion_equals_bruteforce(n, b, tau, sym):
    A = rng_matrix(n, 2, sym)
    B = rng_matrix(n, 3, sym, decay=0.7)
    TA, TB = oracle.Tree(A, b), oracle.Tree(B, b)
    rec = oracle.spamm(TA, TB, tau, triples=True, product=False)["triples"]
    flat_c = oracle.triples_flat(TA, TB, tau)
    flat_np = brute_triples_numpy(TA.norm2(TA.kmax), TB.norm2(TB.kmax), tau)
    assert np.array_equal(oracle.sort_triples(rec), flat_c)
    assert np.array_equal(flat_c, flat_np)
    assert 0 < len(rec) < TA.NB ** 3


def test_tau_zero_all_triples_and_naive_product():
    n, b = 192, 16
    A, B = rng_matrix(n, 4), rng_matrix(n, 5)
    TA, TB = oracle.Tree(A, b), oracle.Tree(B, b)
    r = oracle.spamm(TA, TB, 0.0, triples=True)
    assert r["count"] == TA.NB ** 3   # nothing is culled at tau = 0, not even padding
    ref = A @ B
    err = np.linalg.norm(r["C"] - ref)
    # norm-wise round-off bound of the form of Eq. 5
    assert err <= n * EPS * np.linalg.norm(A) * np.linalg.norm(B)
    naive = oracle.matmul_naive(A, B)
    assert np.linalg.norm(naive - ref) <= n * EPS * np.linalg.norm(A) * np.linalg.norm(B)


def test_root_cull_gives_zero():
    # ||A|| ||B|| < tau: no work is done and C~ = 0, error < tau
    A = rng_matrix(64, 6) * 1e-3
    TA = oracle.Tree(A, 8)
    root = np.sqrt(TA.norm2(0)[0, 0]) ** 2
    r = oracle.spamm(TA, TA, root * 1.0000001, triples=True, stats=True)
    assert r["count"] == 0 and np.all(r["C"] == 0)
    assert r["stats"].tested == [1] + [0] * TA.kmax
    assert np.linalg.norm(A @ A) < root * 1.0000001


def test_equality_survives():
    # strict '<': a product equal to tau is kept. I_{4x4} block norm 2, ones block 4.
    n, b = 16, 4
    A, B = np.eye(n), np.ones((n, n))
    TA, TB = oracle.Tree(A, b), oracle.Tree(B, b)
    r = oracle.spamm(TA, TB, 8.0, triples=True)
    assert r["count"] == 16 and np.array_equal(r["C"], B)
    r = oracle.spamm(TA, TB, np.nextafter(8.0, 9.0), triples=True)
    assert r["count"] == 0


@pytest.mark.parametrize("n,b", [(128, 16), (100, 16)])
def test_identity_operand(n, b):
    B = rng_matrix(n, 7, decay=0.9)
    TI, TB = oracle.Tree(np.eye(n), b), oracle.Tree(B, b)
    nI2, _, NB = blocks_norm2_numpy(np.eye(n), b)
    nB2, PB, _ = blocks_norm2_numpy(B, b)
    tau = 0.05
    r = oracle.spamm(TI, TB, tau, triples=True)
    # survivors are exactly the (i, j, i) with ||I_ii|| ||B_ij|| >= tau
    expect = {(i, j, i) for i in range(NB) for j in range(NB)
              if not (np.sqrt(nI2[i, i]) * np.sqrt(nB2[i, j]) < tau)}
    got = {tuple(int(x) for x in t) for t in r["triples"]}
    assert got == expect
    # C~ is B on the surviving blocks, 0 elsewhere, bit for bit
    M = np.zeros_like(PB)
    for i, j, _ in expect:
        M[i * b:(i + 1) * b, j * b:(j + 1) * b] = PB[i * b:(i + 1) * b, j * b:(j + 1) * b]
    assert np.array_equal(r["C"], M[:n, :n])


def test_diagonal_operand_bitwise():
    n, b = 96, 8
    d = np.random.default_rng(8).uniform(0.5, 2.0, n)
    B = rng_matrix(n, 9)
    r = oracle.spamm(oracle.Tree(np.diag(d), b), oracle.Tree(B, b), 0.0)
    assert np.array_equal(r["C"], d[:, None] * B)


def test_block_diagonal_operand():
    n, b = 64, 8
    A = np.zeros((n, n))
    rng = np.random.default_rng(10)
    for i in range(n // b):
        A[i * b:(i + 1) * b, i * b:(i + 1) * b] = rng.normal(size=(b, b))
    B = rng_matrix(n, 11)
    TA, TB = oracle.Tree(A, b), oracle.Tree(B, b)
    r = oracle.spamm(TA, TB, 1e-6, triples=True)
    for i, j, k in r["triples"]:
        assert i == k
    ref = np.zeros_like(B)
    for i, j, k in r["triples"]:
        ref[i * b:(i + 1) * b, j * b:(j + 1) * b] = (
            A[i * b:(i + 1) * b, i * b:(i + 1) * b] @ B[i * b:(i + 1) * b, j * b:(j + 1) * b])
    np.testing.assert_allclose(r["C"], ref, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("n,b,sym", [(256, 16, False), (240, 32, True), (72, 8, False)])
def test_bruteforce_product_small(n, b, sym):
    A, B = rng_matrix(n, 12, sym), rng_matrix(n, 13, sym)
    TA, TB = oracle.Tree(A, b), oracle.Tree(B, b)
    for tau in (1e-5, 1e-3, 1e-1):
        r = oracle.spamm(TA, TB, tau)
        _, PA, _ = blocks_norm2_numpy(A, b)
        _, PB, _ = blocks_norm2_numpy(B, b)
        trip = brute_triples_numpy(TA.norm2(TA.kmax), TB.norm2(TB.kmax), tau)
        ref = spamm_numpy_from_triples(PA, PB, trip, b, n)
        scale = np.linalg.norm(A) * np.linalg.norm(B)
        assert np.linalg.norm(r["C"] - ref) <= 4 * n * EPS * scale


def test_error_bound_and_monotone_count():
    n, b = 256, 16
    A = W.algebraic_decay(n, 2, 0)
    TA = oracle.Tree(A, b)
    exact = A @ A
    prev = None
    for tau in (0.0, 1e-10, 1e-8, 1e-6, 1e-4, 1e-2, 1.0):
        r = oracle.spamm(TA, TA, tau, stats=True)
        err = np.linalg.norm(r["C"] - exact)
        fb = oracle.flat_bound(TA, TA, tau)
        hb = sum(r["stats"].culled_bound)
        slack = 4 * n * EPS * np.linalg.norm(A) ** 2
        assert err <= fb + slack and err <= hb + slack
        if prev is not None:
            assert r["count"] <= prev
        prev = r["count"]


def test_error_is_order_tau():
    # Sec. III: SpAMM error is O(tau); check the log-log slope on algebraic decay
    A = W.algebraic_decay(512, 2, 0)
    TA = oracle.Tree(A, 16)
    exact = A @ A
    taus = np.array([1e-9, 1e-8, 1e-7, 1e-6])
    errs = np.array([np.linalg.norm(oracle.spamm(TA, TA, t)["C"] - exact) for t in taus])
    slope = np.polyfit(np.log10(taus), np.log10(errs), 1)[0]
    assert 0.6 < slope < 1.4, slope


def test_block_evaluation_matches_full():
    A = W.exp_decay(300, 0.85, 1, 0)
    TA = oracle.Tree(A, 32)
    full = oracle.spamm(TA, TA, 1e-8)["C"]
    P = np.zeros((TA.NB * 32, TA.NB * 32))
    P[:300, :300] = full
    for i, j in [(0, 0), (3, 4), (9, 9), (9, 0), (5, 5)]:
        blk = oracle.spamm_block(TA, TA, 1e-8, i, j)
        assert np.array_equal(blk, P[i * 32:(i + 1) * 32, j * 32:(j + 1) * 32])


def test_threads_do_not_change_bits():
    if oracle.max_threads() < 2:
        pytest.skip("oracle built without OpenMP")
    A = W.algebraic_decay(512, 2, 0)
    TA = oracle.Tree(A, 16)
    c1 = oracle.spamm(TA, TA, 1e-8, threads=1)["C"]
    c4 = oracle.spamm(TA, TA, 1e-8, threads=4)["C"]
    assert np.array_equal(c1, c4)


def test_fig1_golden_counts():
    import json, os
    path = os.path.join(os.path.dirname(__file__), "golden", "fig1_counts.json")
    gold = json.load(open(path))
    for case in gold["cases"]:
        A, B = W.fig1_pair(case["pair"], case["n"])
        TA, TB = oracle.Tree(A, case["leaf"]), oracle.Tree(B, case["leaf"])
        r = oracle.spamm(TA, TB, case["tau"], product=False, stats=True)
        assert r["count"] == case["leaf_triples"]
        assert r["stats"].tested == case["tested"]
        assert r["stats"].culled == case["culled"]


# ---------------------------------------------------------------- planted mistakes

def _pins_fail(L):
    """Run a handful of pins against an oracle library; True when one of them fails."""
    def tree(A, b):
        return oracle.Tree(A, b, L)
    try:
        # norms: closed form of a constant matrix
        T = tree(np.full((32, 32), 2.0), 8)
        for l in range(T.kmax + 1):
            if not np.all(T.norm2(l) == 4.0 * 64 * 4 ** (T.kmax - l)):
                return True
        # strict inequality at equality
        TI, TO = tree(np.eye(16), 4), tree(np.ones((16, 16)), 4)
        if oracle.spamm(TI, TO, 8.0)["count"] != 16:
            return True
        # tau = 0 against numpy, non-symmetric operands
        A, B = rng_matrix(64, 21), rng_matrix(64, 22)
        TA, TB = tree(A, 8), tree(B, 8)
        r = oracle.spamm(TA, TB, 0.0)
        if np.linalg.norm(r["C"] - A @ B) > 64 * EPS * np.linalg.norm(A) * np.linalg.norm(B):
            return True
        # recursion against numpy brute force, non-symmetric operands
        A, B = rng_matrix(128, 23), np.triu(rng_matrix(128, 24, decay=0.6))
        TA, TB = tree(A, 8), tree(B, 8)
        rec = oracle.spamm(TA, TB, 1e-3, triples=True, product=False)["triples"]
        nA2, _, _ = blocks_norm2_numpy(A, 8)
        nB2, _, _ = blocks_norm2_numpy(B, 8)
        if not np.array_equal(oracle.sort_triples(rec), brute_triples_numpy(nA2, nB2, 1e-3)):
            return True
        # the depth-scaled threshold against numpy brute force over every tier
        A, B = rng_matrix(128, 25), rng_matrix(128, 26, decay=0.7)
        TA, TB = tree(A, 8), tree(B, 8)
        rec = oracle.spamm(TA, TB, DEPTH_TAU, triples=True, product=False, depth_scaled=True)["triples"]
        if not np.array_equal(oracle.sort_triples(rec), brute_depth_triples_numpy(A, B, 8, DEPTH_TAU)):
            return True
    except Exception:
        return True
    return False


def test_pins_pass_on_oracle():
    assert not _pins_fail(oracle.lib())


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6, 7])
def test_pins_catch_planted_mistake(mutant):
    L = oracle.mutant_lib(mutant)
    assert L.oracle_mutant() == mutant
    assert _pins_fail(L)


# ---------------------------------------------------------------- operand formats

def test_format_rounding_matches_torch_on_float_inputs():
    # on FP32-representable inputs a single rounding to BF16 / FP16 is what torch does
    torch = pytest.importorskip("torch")
    from oracle import formats as F
    r = np.random.default_rng(3)
    x = (r.standard_normal(20000) * np.exp(r.uniform(-30, 10, 20000))).astype(np.float32).astype(np.float64)
    assert np.array_equal(F.round_to(x, "bf16"), torch.tensor(x).to(torch.bfloat16).double().numpy())
    assert np.array_equal(F.round_to(x, "fp16"), torch.tensor(x).to(torch.float16).double().numpy())


def test_format_rounding_hand_cases():
    from oracle import formats as F
    # ties go to even; just above a tie rounds up (single rounding from FP64)
    assert F.round_to(np.array([1 + 2.0 ** -8]), "bf16")[0] == 1.0
    assert F.round_to(np.array([1 + 3 * 2.0 ** -8]), "bf16")[0] == 1 + 2.0 ** -6
    assert F.round_to(np.array([1 + 2.0 ** -8 + 2.0 ** -40]), "bf16")[0] == 1 + 2.0 ** -7
    assert F.round_to(np.array([1 + 2.0 ** -11]), "tf32")[0] == 1.0
    assert F.round_to(np.array([1 + 2.0 ** -11 + 2.0 ** -45]), "tf32")[0] == 1 + 2.0 ** -10
    assert F.round_to(np.array([2.0 ** -25]), "fp16")[0] == 0.0           # half of the least subnormal
    assert F.round_to(np.array([3 * 2.0 ** -25]), "fp16")[0] == 2.0 ** -23
    assert F.round_to(np.array([65504.0]), "fp16")[0] == 65504.0
    hi, lo = F.split_bf16(np.array([np.pi]))
    assert abs(hi[0] + lo[0] - np.pi) < 2.0 ** -16 * np.pi
    # TF32 split: 1 + 2^-11 + 2^-30 lies just above the tie between 1 and 1 + 2^-10, so
    # hi = 1 + 2^-10 and the remainder -2^-11 + 2^-30 rounds to -2^-11 in 11 bits
    hi, lo = F.split(np.array([1 + 2.0 ** -11 + 2.0 ** -30]), "tf32")
    assert hi[0] == 1 + 2.0 ** -10 and lo[0] == -2.0 ** -11
    x = np.random.default_rng(5).normal(size=1000) * 10.0 ** np.random.default_rng(6).uniform(-20, 20, 1000)
    hi, lo = F.split(x, "tf32")
    assert np.all(np.abs(hi + lo - x) <= 2.0 ** -22 * np.abs(x))
    assert np.array_equal(F.round_to(hi, "tf32"), hi) and np.array_equal(F.round_to(lo, "tf32"), lo)


def test_values_oracle_uses_substituted_leaves():
    # same triple list as the plain product; leaf values from the second pair
    A = rng_matrix(160, 31)
    TA = oracle.Tree(A, 16)
    T2 = oracle.Tree(2.0 * A, 16)
    plain = oracle.spamm(TA, TA, 1e-4)["C"]
    twice = oracle.spamm_values(TA, TA, T2, TA, 1e-4)
    assert np.array_equal(twice, 2.0 * plain)
    blk = oracle.spamm_block(TA, TA, 1e-4, 3, 4, T2, TA)
    assert np.array_equal(blk, 2.0 * plain[48:64, 64:80])


# ---------------------------------------------------------------- depth-scaled threshold

def test_depth_pin_has_no_near_ties():
    # the depth-scaled pin compares two summation orders of the norms: no tested product
    # may lie within 1e-6 of its tier's threshold
    _, gap = brute_depth_triples_numpy(rng_matrix(128, 25), rng_matrix(128, 26, decay=0.7), 8, DEPTH_TAU, True)
    assert gap > 1e-6


@pytest.mark.parametrize("seed,leaf,tau", [(41, 8, 1e-2), (42, 16, 1e-3), (43, 4, 3e-2)])
def test_depth_scaled_error_is_rigorous(seed, leaf, tau):
    # Sec. II: with tau^{k+1} = tau^k / 8 every dropped sub-product of tier k is below
    # tau 8^-k and tier k holds at most 8^k of them, so ||C~ - AB||_F < (kmax + 1) tau
    A, B = rng_matrix(160, seed, decay=0.85), rng_matrix(160, seed + 100, decay=0.85)
    TA, TB = oracle.Tree(A, leaf), oracle.Tree(B, leaf)
    r = oracle.spamm(TA, TB, tau, depth_scaled=True, stats=True)
    err = np.linalg.norm(r["C"] - A @ B)
    assert err < (TA.kmax + 1) * tau
    # tier k's culled products each stay below its threshold: their sum bounds the error
    assert err <= sum(r["stats"].culled_bound) * (1 + 1e-12)
    # the depth-scaled survivors include the plain ones (every threshold is <= tau)
    plain = oracle.sort_triples(oracle.spamm(TA, TB, tau, triples=True, product=False)["triples"])
    deep = oracle.sort_triples(oracle.spamm(TA, TB, tau, triples=True, product=False, depth_scaled=True)["triples"])
    assert len(deep) >= len(plain)
    assert {tuple(t) for t in plain} <= {tuple(t) for t in deep}

