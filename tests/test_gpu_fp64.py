"""GPU parity of the FP64 SpAMM path against the CPU oracle, through the C ABI.

Bars: norms of every tier within 1e-13 relative and monotone bit for bit; the
surviving leaf triples identical outside the 1e-12 near-tau band; C within 1e-12
relative Frobenius error at equal tau; tier counters identical.
"""
import numpy as np
import pytest

import oracle
from parity import adjust_for_band, compare_triples, rel_fro
from paper_1011_3534_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


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


def rng_matrix(n, seed, decay=0.8, sym=False):
    r = np.random.default_rng(seed)
    d = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :])
    M = r.uniform(-1, 1, (n, n)) * decay ** d
    return (M + M.T) / 2 if sym else M


def run_case(S, ctx, A, B, leaf, tau, host=False, threads=8):
    n = A.shape[0]
    fl = S.SPAMM_KEEP_FP64
    if host:
        tA = S.spamm_tree_build(ctx, A, n, leaf, fl)
        tB = S.spamm_tree_build(ctx, B, n, leaf, fl)
    else:
        tA = S.spamm_tree_build(ctx, torch.from_numpy(A).cuda(), n, leaf, fl)
        tB = S.spamm_tree_build(ctx, torch.from_numpy(B).cuda(), n, leaf, fl)
    tC = S.spamm_multiply(ctx, tA, tB, tau, S.SPAMM_FP64)
    out = dict(C=S.spamm_tree_to_dense(tC), trip=S.spamm_triples(tC), stats=S.spamm_stats(tC),
               normsA=[S.spamm_tree_norms(tA, l) for l in range(tA.kmax + 1)],
               normsC=[S.spamm_tree_norms(tC, l) for l in range(tC.kmax + 1)], NB=tA.NB)
    for t in (tC, tB, tA):
        S.spamm_tree_free(t)
    return out


def check_against_oracle(A, B, leaf, tau, g, full_c=True):
    TA, TB = oracle.Tree(A, leaf), oracle.Tree(B, leaf)
    ref = oracle.spamm(TA, TB, tau, triples=True, stats=True, product=False)
    NB = TA.NB
    assert g["NB"] == NB
    # norms of every tier of A
    for l in range(TA.kmax + 1):
        o = TA.norm2(l)
        np.testing.assert_allclose(g["normsA"][l], o, rtol=1e-13, atol=0)
    nA2, nB2 = TA.norm2(TA.kmax), TB.norm2(TB.kmax)
    only_g, only_o = compare_triples(g["trip"], oracle.sort_triples(ref["triples"]), NB, nA2, nB2, tau)
    st = g["stats"]
    if not len(only_g) and not len(only_o):
        assert st["tested"] == ref["stats"].tested
        assert st["culled"] == ref["stats"].culled
        assert st["leaf_products"] == ref["count"]
        np.testing.assert_allclose(st["culled_bound"], ref["stats"].culled_bound, rtol=1e-11, atol=1e-300)
    if full_c:
        Cref = oracle.spamm(TA, TB, tau, threads=oracle.max_threads())["C"]
        Cref = adjust_for_band(Cref, A, B, leaf, NB, only_g, only_o)
        err = rel_fro(g["C"], Cref)
        assert err <= 1e-12, err
    return TA, TB


def check_pyramid_monotone(norms):
    for l in range(len(norms) - 1):
        par, ch = norms[l], norms[l + 1]
        for a in range(2):
            for c in range(2):
                assert np.all(par >= ch[a::2, c::2])


@pytest.mark.parametrize("n,leaf,tau,kind", [
    (1000, 32, 1e-8, "exp"),      # ragged tail: 1000 = 31 * 32 + 8
    (777, 16, 1e-6, "alg"),
    (3000, 64, 1e-8, "alg"),
    (4100, 128, 1e-6, "exp"),
    (2048, 64, 0.0, "exp"),       # tau = 0: every padded triple survives
    (1536, 16, 1e-4, "rand"),
])
def test_fp64_parity(S, ctx, n, leaf, tau, kind):
    if kind == "exp":
        A = W.exp_decay(n, 0.85, 1, 0)
    elif kind == "alg":
        A = W.algebraic_decay(n, 2, 0)
    else:
        A = rng_matrix(n, 5, 0.9, sym=True)
    g = run_case(S, ctx, A, A, leaf, tau)
    check_against_oracle(A, A, leaf, tau, g)
    check_pyramid_monotone(g["normsA"])
    check_pyramid_monotone(g["normsC"])


def test_fp64_nonsymmetric_pair(S, ctx):
    n, leaf, tau = 900, 32, 1e-5
    A = rng_matrix(n, 11, 0.85)
    B = np.triu(rng_matrix(n, 12, 0.9))
    g = run_case(S, ctx, A, B, leaf, tau)
    check_against_oracle(A, B, leaf, tau, g)


def test_workload_exp1024(S, ctx):
    # n = 1024 exponential decay 0.85^|i-j|, leaf 32, tau = 1e-8
    A = W.exp_decay(1024, 0.85, 1, 0)
    g = run_case(S, ctx, A, A, 32, 1e-8)
    check_against_oracle(A, A, 32, 1e-8, g)


@pytest.mark.parametrize("n,leaf", [(1, 16), (20, 32), (64, 64), (65, 64), (129, 128)])
def test_small_and_degenerate(S, ctx, n, leaf):
    A = rng_matrix(n, 3, 0.7)
    for tau in (0.0, 1e-3):
        g = run_case(S, ctx, A, A, leaf, tau)
        check_against_oracle(A, A, leaf, tau, g)


def test_root_cull_empty(S, ctx):
    A = rng_matrix(256, 4) * 1e-3
    g = run_case(S, ctx, A, A, 16, 1e6)
    assert len(g["trip"]) == 0 and np.all(g["C"] == 0)
    assert g["stats"]["tested"][0] == 1 and g["stats"]["culled"][0] == 1


def test_identity_and_diagonal_bitwise(S, ctx):
    n, leaf = 640, 64
    B = rng_matrix(n, 6, 0.9)
    g = run_case(S, ctx, np.eye(n), B, leaf, 0.0)
    assert np.array_equal(g["C"], B)
    d = np.random.default_rng(7).uniform(0.5, 2.0, n)
    g = run_case(S, ctx, np.diag(d), B, leaf, 0.0)
    assert np.array_equal(g["C"], d[:, None] * B)


def test_host_input_and_determinism(S, ctx):
    A = W.algebraic_decay(2000, 2, 0)
    g1 = run_case(S, ctx, A, A, 64, 1e-7, host=True)
    g2 = run_case(S, ctx, A, A, 64, 1e-7, host=False)
    assert np.array_equal(g1["C"], g2["C"])
    assert np.array_equal(g1["trip"], g2["trip"])
    assert g1["stats"]["culled_bound"] == g2["stats"]["culled_bound"]


def test_invalid_arguments(S, ctx):
    A = torch.zeros((100, 100), dtype=torch.float64, device="cuda")
    with pytest.raises(S.SpammError) as e:
        S.spamm_tree_build(ctx, A, 100, 48, S.SPAMM_KEEP_FP64)
    assert e.value.status == S.SPAMM_EINVAL
    t = S.spamm_tree_build(ctx, A, 100, 16, S.SPAMM_KEEP_FP64)
    u = S.spamm_tree_build(ctx, A, 100, 32, S.SPAMM_KEEP_FP64)
    with pytest.raises(S.SpammError):
        S.spamm_multiply(ctx, t, u, 1e-3)
    with pytest.raises(S.SpammError):
        S.spamm_multiply(ctx, t, t, -1.0)
    with pytest.raises(S.SpammError):
        S.spamm_multiply(ctx, t, t, float("nan"))
    with pytest.raises(S.SpammError):
        S.spamm_multiply(ctx, t, t, 1e-3, S.SPAMM_BF16)   # no BF16 copy, leaf 16
    S.spamm_tree_free(t)
    S.spamm_tree_free(u)


@pytest.mark.parametrize("tau", [1e-10, 1e-8, 1e-6, 1e-4])
def test_workload_alg8192_fp64_sampled(S, ctx, tau):
    # n = 8192 algebraic decay, leaf 64: full triple list; C on sampled output blocks
    n, leaf = 8192, 64
    A = W.algebraic_decay(n, 2, 0)
    g = run_case(S, ctx, A, A, leaf, tau)
    TA, _ = check_against_oracle(A, A, leaf, tau, g, full_c=False)
    rng = np.random.default_rng(7)
    NB = TA.NB
    blocks = [(0, 0), (0, NB - 1), (NB - 1, NB - 1), (5, 6)] + [tuple(x) for x in rng.integers(0, NB, (12, 2))]
    for i, j in blocks:
        ref = oracle.spamm_block(TA, TA, tau, int(i), int(j))
        got = g["C"][i * leaf:(i + 1) * leaf, j * leaf:(j + 1) * leaf]
        d = np.linalg.norm(got - ref)
        assert d <= 1e-12 * max(np.linalg.norm(ref), 1e-300) or d == 0, (i, j, d)


@pytest.mark.parametrize("n,leaf,tau,kind", [(1000, 32, 1e-8, "exp"), (3000, 64, 1e-8, "alg"), (1536, 16, 1e-4, "rand"),
                                             (2048, 64, 0.0, "exp")])
def test_fp64_symmetric_product(S, ctx, n, leaf, tau, kind):
    # SPAMM_SYM_PRODUCT: blocks i <= j multiplied, the rest mirrored; same triples (the
    # cull reads a symmetric tree's norms on and above the diagonal) and C within 1e-12 of
    # the oracle
    A = {"exp": lambda: W.exp_decay(n, 0.85, 1, 0), "alg": lambda: W.algebraic_decay(n, 2, 0),
         "rand": lambda: rng_matrix(n, 5, 0.9, sym=True)}[kind]()
    fl = S.SPAMM_KEEP_FP64 | S.SPAMM_SYMMETRIC
    tA = S.spamm_tree_build(ctx, torch.from_numpy(A).cuda(), n, leaf, fl)
    tC = S.spamm_multiply(ctx, tA, tA, tau, S.SPAMM_FP64, S.SPAMM_SYM_PRODUCT)
    C, trip, st = S.spamm_tree_to_dense(tC), S.spamm_triples(tC), S.spamm_stats(tC)
    norms = [S.spamm_tree_norms(tA, l) for l in range(tA.kmax + 1)]
    normsC = [S.spamm_tree_norms(tC, l) for l in range(tC.kmax + 1)]
    S.spamm_tree_free(tC)
    S.spamm_tree_free(tA)
    for nl in norms + normsC:
        np.testing.assert_allclose(nl, nl.T, rtol=1e-11, atol=0)
    check_pyramid_monotone(norms)
    check_pyramid_monotone(normsC)
    assert np.array_equal(C, C.T)
    TA = oracle.Tree(A, leaf)
    ref = oracle.spamm(TA, TA, tau, triples=True, product=False)
    only_g, only_o = compare_triples(trip, oracle.sort_triples(ref["triples"]), TA.NB, TA.norm2(TA.kmax),
                                     TA.norm2(TA.kmax), tau)
    assert st["leaf_products"] + st["mirrored_products"] == ref["count"] + len(only_g) - len(only_o)
    assert st["mirrored_products"] <= st["leaf_products"]
    Cref = oracle.spamm(TA, TA, tau, threads=oracle.max_threads())["C"]
    Cref = adjust_for_band(Cref, A, A, leaf, TA.NB, only_g, only_o)
    assert rel_fro(C, Cref) <= 1e-12


def test_page_locked_host_buffers(S, ctx):
    """Host input in page-locked memory goes in on the context's input copy stream,
    pageable input through the staging buffer; dense output is written synchronously or
    asynchronously (complete after spamm_sync). All give the same tree, product and
    dense output, bit for bit, for a ragged order and both precision classes."""
    n = 1000
    A = W.algebraic_decay(n, 2, 3)
    A_pin = torch.from_numpy(A).pin_memory()
    for prec, leaf, fl in ((S.SPAMM_FP64, 32, S.SPAMM_KEEP_FP64),
                           (S.SPAMM_BF16, 64, S.COPY_FLAG[S.SPAMM_BF16] | S.SPAMM_SYMMETRIC)):
        outs = []
        for src in (A, A_pin.numpy()):
            t = S.spamm_tree_build(ctx, src, n, leaf, fl)
            S.spamm_tree_update(t, src)
            c = S.spamm_multiply(ctx, t, t, 1e-9, prec)
            dense_pageable = S.spamm_tree_to_dense(c)
            C_pin = torch.empty((n, n), dtype=torch.float64).pin_memory()
            S.spamm_tree_to_dense(c, C_pin.numpy())
            # asynchronous output, overlapped with a rebuild of the input, complete after sync
            C_async = torch.full((n, n), np.nan, dtype=torch.float64).pin_memory()
            S.spamm_tree_to_dense(c, C_async.numpy(), asynchronous=True)
            S.spamm_tree_update(t, src)
            S.spamm_sync(ctx)
            assert np.array_equal(C_async.numpy(), C_pin.numpy())
            outs.append((S.spamm_tree_norms(t, t.kmax), dense_pageable, C_pin.numpy().copy()))
            S.spamm_tree_free(c)
            S.spamm_tree_free(t)
        (n0, d0, p0), (n1, d1, p1) = outs
        assert np.array_equal(n0, n1)
        assert np.array_equal(d0, d1) and np.array_equal(d0, p0) and np.array_equal(d0, p1)


@pytest.mark.parametrize("n,leaf,tau,prec_name,sym", [(1000, 32, 1e-6, "fp64", False), (2048, 64, 1e-4, "fp64", True),
                                                      (3000, 64, 1e-5, "bf16", True), (1536, 128, 1e-3, "bf16", False)])
def test_depth_scaled_threshold(S, ctx, n, leaf, tau, prec_name, sym):
    # SPAMM_DEPTH_TAU: tier k tests against tau 8^-k (Sec. II); the surviving triples,
    # tier counts and culled bounds equal the oracle's depth-scaled recursion, C equals
    # it within the FP64 bar (FP64) or the BF16 sanity bar, and the rigorous bound holds
    A = W.algebraic_decay(n, 2, 4)
    prec = S.PRECISIONS[prec_name]
    fl = (S.SPAMM_KEEP_FP64 if prec == S.SPAMM_FP64 else S.COPY_FLAG[prec]) | (S.SPAMM_SYMMETRIC if sym else 0)
    tA = S.spamm_tree_build(ctx, torch.from_numpy(A).cuda(), n, leaf, fl)
    flags = S.SPAMM_DEPTH_TAU | (S.SPAMM_SYM_PRODUCT if sym else 0)
    tC = S.spamm_multiply(ctx, tA, tA, tau, prec, flags)
    C, trip, st = S.spamm_tree_to_dense(tC), S.spamm_triples(tC), S.spamm_stats(tC)
    S.spamm_tree_free(tC)
    S.spamm_tree_free(tA)
    TA = oracle.Tree(A, leaf)
    ref = oracle.spamm(TA, TA, tau, triples=True, stats=True, product=False, depth_scaled=True)
    assert np.array_equal(oracle.sort_triples(trip), oracle.sort_triples(ref["triples"]))
    if not sym:
        assert st["tested"] == ref["stats"].tested and st["culled"] == ref["stats"].culled
        np.testing.assert_allclose(st["culled_bound"], ref["stats"].culled_bound, rtol=1e-11, atol=1e-300)
    C64 = oracle.spamm(TA, TA, tau, threads=oracle.max_threads(), depth_scaled=True)["C"]
    err = rel_fro(C, C64)
    assert err < (1e-12 if prec_name == "fp64" else 1e-2)
    exact = A @ A
    assert np.linalg.norm(C64 - exact) < (TA.kmax + 1) * tau
    plain = oracle.spamm(TA, TA, tau, product=False)["count"]
    print(f"depth-scaled tau {tau} {prec_name} leaf {leaf}: {ref['count']} triples (plain {plain}), "
          f"error {np.linalg.norm(C64 - exact):.2e} < {(TA.kmax + 1) * tau:.2e}")
