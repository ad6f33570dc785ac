"""Batched products (one persistent tensor-core launch over all products, optionally a
CUDA graph) against the single-product path, and the leaf-size autotuner.

Each product of a batch runs the same per-item arithmetic in the same order as when it
is multiplied alone, so its C must be identical bit for bit; the triple lists equal.
"""
import numpy as np
import pytest

import oracle
from parity import compare_triples
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
    st = torch.cuda.Stream()
    c = S.spamm_ctx_create(0, st)
    c.stream = st
    yield c
    S.spamm_ctx_destroy(c)


def batch_inputs(count, seed=3):
    shapes = W.batched_shapes(count=count, lo=512, hi=3072, seed=seed)
    return [W.batched_matrix(m, n, lam, seed=seed) for m, (n, lam) in enumerate(shapes)]


def build(S, ctx, mats, leaves, prec):
    fl = S.COPY_FLAG[prec] | S.SPAMM_SYMMETRIC | (S.SPAMM_NO_RIGHT if prec != S.SPAMM_FP64 else 0)
    with torch.cuda.stream(ctx.stream):
        return [S.spamm_tree_build(ctx, torch.from_numpy(M).cuda(), M.shape[0], b, fl) for M, b in zip(mats, leaves)]


@pytest.mark.parametrize("prec_name", ["bf16", "bf16x3", "fp64"])
def test_batched_equals_single(S, ctx, prec_name):
    prec = S.PRECISIONS[prec_name]
    mats = batch_inputs(12)
    leaves = [64 if i % 3 else 128 for i in range(len(mats))] if prec != S.SPAMM_FP64 else [32, 64] * 6
    trees = build(S, ctx, mats, leaves, prec)
    taus = [1e-7 * (1 + (i % 4)) for i in range(len(mats))]
    Cb = S.spamm_multiply_batched(ctx, trees, trees, taus, prec)
    for p, (t, tau) in enumerate(zip(trees, taus)):
        Cs = S.spamm_multiply(ctx, t, t, tau, prec)
        assert np.array_equal(S.spamm_triples(Cb[p]), S.spamm_triples(Cs)), p
        assert np.array_equal(S.spamm_tree_to_dense(Cb[p]), S.spamm_tree_to_dense(Cs)), p
        sb, ss = S.spamm_stats(Cb[p]), S.spamm_stats(Cs)
        assert sb["leaf_products"] == ss["leaf_products"] and sb["mma_flops"] == ss["mma_flops"]
        S.spamm_tree_free(Cs)
    # the triples are the oracle's (one product checked against the CPU)
    T = oracle.Tree(mats[0], leaves[0])
    ref = oracle.spamm(T, T, taus[0], triples=True, product=False)
    compare_triples(S.spamm_triples(Cb[0]), oracle.sort_triples(ref["triples"]), T.NB, T.norm2(T.kmax),
                    T.norm2(T.kmax), taus[0])
    for t in Cb + trees:
        S.spamm_tree_free(t)


def test_batched_graph_replay(S, ctx):
    prec = S.SPAMM_BF16
    mats = batch_inputs(8, seed=5)
    trees = build(S, ctx, mats, [64] * len(mats), prec)
    C = None
    for tau in (1e-7, 1e-5, 1e-7):
        taus = [tau] * len(mats)
        C = S.spamm_multiply_batched(ctx, trees, trees, taus, prec, S.SPAMM_GRAPH, C)
        for p, t in enumerate(trees):
            Cs = S.spamm_multiply(ctx, t, t, tau, prec)
            assert np.array_equal(S.spamm_tree_to_dense(C[p]), S.spamm_tree_to_dense(Cs)), (tau, p)
            assert S.spamm_stats(C[p])["leaf_products"] == S.spamm_stats(Cs)["leaf_products"]
            S.spamm_tree_free(Cs)
    for t in C + trees:
        S.spamm_tree_free(t)


def test_tuner_picks_a_supported_leaf(S, ctx):
    M = W.batched_matrix(0, 2048, 0.85)
    with torch.cuda.stream(ctx.stream):
        d = torch.from_numpy(M).cuda()
        leaf, ms = S.spamm_tune_leaf(ctx, d, 2048, 1e-7, S.SPAMM_BF16, S.SPAMM_SYMMETRIC)
        assert leaf in (16, 32, 64, 128) and ms > 0
        leaf2, ms2 = S.spamm_tune_leaf(ctx, d, 2048, 1e-7, S.SPAMM_BF16, S.SPAMM_SYMMETRIC)
        assert (leaf2, ms2) == (leaf, ms)   # cached
        leaf3, _ = S.spamm_tune_leaf(ctx, d, 2048, 1e-7, S.SPAMM_FP64, S.SPAMM_SYMMETRIC)
        assert leaf3 in (16, 32, 64, 128)


def test_batched_update_equals_single_updates(S, ctx):
    # the rebuilds spread over the side streams give the same trees as one by one: the
    # same norms on every tier and the same products, bit for bit
    mats = batch_inputs(10, seed=5)
    prec = S.SPAMM_BF16
    leaves = [64 if i % 2 else 128 for i in range(len(mats))]
    a = build(S, ctx, mats, leaves, prec)
    b = build(S, ctx, mats, leaves, prec)
    with torch.cuda.stream(ctx.stream):
        dev = [torch.from_numpy(2.0 * M).cuda() for M in mats]
        for t, X in zip(a, dev):
            S.spamm_tree_update(t, X)
        S.spamm_tree_update_batched(ctx, b, dev)
    for ta, tb in zip(a, b):
        for l in range(ta.kmax + 1):
            assert np.array_equal(S.spamm_tree_norms(ta, l), S.spamm_tree_norms(tb, l))
        ca = S.spamm_multiply(ctx, ta, ta, 1e-6, prec)
        cb = S.spamm_multiply(ctx, tb, tb, 1e-6, prec)
        assert np.array_equal(S.spamm_tree_to_dense(ca), S.spamm_tree_to_dense(cb))
        S.spamm_tree_free(ca)
        S.spamm_tree_free(cb)
    for t in a + b:
        S.spamm_tree_free(t)



def test_batched_config4_against_oracle(S, ctx):
    # config-4 shapes (256 symmetric exponential-decay matrices, n log-uniform in
    # [512, 8192], seed 3): five products spanning n, the largest n = 8192 among them,
    # leaf 128 BF16 (the tuner's pick for this batch), one persistent launch from a
    # CUDA graph captured at another tau and replayed at tau = 1e-7. Every product's
    # triple list against the oracle's, and C on sampled output blocks against the
    # oracle with BF16-rounded leaf operands under the FP32 bound of test_gpu_tc.py
    from oracle import formats as F
    from parity import tc_bound
    shapes = W.batched_shapes()
    order = sorted(range(len(shapes)), key=lambda m: shapes[m][0])
    pick = [order[0], order[len(order) // 4], order[len(order) // 2], order[3 * len(order) // 4], order[-1]]
    assert shapes[pick[-1]][0] == 8192
    mats = [W.batched_matrix(m, *shapes[m]) for m in pick]
    leaf, tau, prec = 128, 1e-7, S.SPAMM_BF16
    trees = build(S, ctx, mats, [leaf] * len(mats), prec)
    C = S.spamm_multiply_batched(ctx, trees, trees, [1e-5] * len(mats), prec, S.SPAMM_GRAPH)
    C = S.spamm_multiply_batched(ctx, trees, trees, [tau] * len(mats), prec, S.SPAMM_GRAPH, C)
    rng = np.random.default_rng(7)
    for p, M in enumerate(mats):
        T = oracle.Tree(M, leaf)
        ref = oracle.spamm(T, T, tau, triples=True, product=False)
        only_g, only_o = compare_triples(S.spamm_triples(C[p]), oracle.sort_triples(ref["triples"]), T.NB,
                                         T.norm2(T.kmax), T.norm2(T.kmax), tau)
        assert not len(only_g) and not len(only_o)
        cnt = np.zeros((T.NB, T.NB), dtype=np.int64)
        np.add.at(cnt, (ref["triples"][:, 0], ref["triples"][:, 1]), 1)
        Mr = F.round_to(M, "bf16")
        tR, tAbs = oracle.Tree(Mr, leaf), oracle.Tree(np.abs(Mr), leaf)
        nb = -(-M.shape[0] // leaf)
        blocks = [(0, 0), (0, nb - 1), (nb - 1, nb - 1)] + [tuple(int(v) for v in x) for x in rng.integers(0, nb, (6, 2))]
        got_all = S.spamm_tree_to_dense(C[p])
        for i, j in blocks:
            Cref = oracle.spamm_block(T, T, tau, i, j, tR, tR)
            Cabs = oracle.spamm_block(T, T, tau, i, j, tAbs, tAbs)
            got = np.zeros((leaf, leaf))
            blk = got_all[i * leaf:(i + 1) * leaf, j * leaf:(j + 1) * leaf]
            got[:blk.shape[0], :blk.shape[1]] = blk
            bound = tc_bound(leaf * cnt[i, j], "bf16", Cabs)
            assert np.all(np.abs(got - Cref) <= bound), (p, i, j)
    for t in C + trees:
        S.spamm_tree_free(t)


def test_shape_tuner_returns_a_runnable_shape(S, ctx):
    # (leaf, tile-shape flags) over leaf 16/32 warp tiles, leaf 64 tcgen05 items and warp
    # tiles, leaf 128 items; the chosen pair runs, and a second call is served from the cache
    M = W.batched_matrix(0, 2048, 0.85)
    with torch.cuda.stream(ctx.stream):
        d = torch.from_numpy(M).cuda()
        leaf, tf, ms = S.spamm_tune_shape(ctx, d, 2048, 1e-7, S.SPAMM_TF32X3, S.SPAMM_SYMMETRIC)
        assert leaf in (16, 32, 64, 128) and tf in (0, S.SPAMM_WARP_TILES) and ms > 0
        assert tf == 0 or leaf == 64
        assert S.spamm_tune_shape(ctx, d, 2048, 1e-7, S.SPAMM_TF32X3, S.SPAMM_SYMMETRIC) == (leaf, tf, ms)
        t = S.spamm_tree_build(ctx, d, 2048, leaf, S.COPY_FLAG[S.SPAMM_TF32X3] | S.SPAMM_SYMMETRIC)
        C = S.spamm_multiply(ctx, t, t, 1e-7, S.SPAMM_TF32X3, tf)
        assert S.spamm_stats(C)["leaf_products"] > 0
        leaf64, tf64, _ = S.spamm_tune_shape(ctx, d, 2048, 1e-7, S.SPAMM_FP64, S.SPAMM_SYMMETRIC)
        assert tf64 == 0 and leaf64 in (16, 32, 64, 128)
        for x in (C, t):
            S.spamm_tree_free(x)


@pytest.mark.parametrize("prec_name", ["bf16", "tf32x3"])
def test_batched_warp_tiles(S, ctx, prec_name):
    # leaf 64 in warp tiles inside a batch equals the single products in the same shape
    # bit for bit; against the tcgen05 items the triples are the same and C agrees to
    # the FP32 accumulation order
    prec = S.PRECISIONS[prec_name]
    mats = batch_inputs(6, seed=9)
    trees = build(S, ctx, mats, [64] * len(mats), prec)
    taus = [1e-7] * len(mats)
    Cb = S.spamm_multiply_batched(ctx, trees, trees, taus, prec, S.SPAMM_WARP_TILES)
    for p, t in enumerate(trees):
        Cs = S.spamm_multiply(ctx, t, t, taus[p], prec, S.SPAMM_WARP_TILES)
        assert np.array_equal(S.spamm_triples(Cb[p]), S.spamm_triples(Cs)), p
        assert np.array_equal(S.spamm_tree_to_dense(Cb[p]), S.spamm_tree_to_dense(Cs)), p
        Ci = S.spamm_multiply(ctx, t, t, taus[p], prec)
        assert np.array_equal(S.spamm_triples(Ci), S.spamm_triples(Cs)), p
        a, b = S.spamm_tree_to_dense(Cs), S.spamm_tree_to_dense(Ci)
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b), p
        for x in (Cs, Ci):
            S.spamm_tree_free(x)
    for t in Cb + trees:
        S.spamm_tree_free(t)
