"""GPU parity of the tensor-core (tcgen05) leaf products against the CPU oracle.

The cull is the FP64 one, so the triple list must equal the oracle's exactly (outside
the near-tau band). C is compared with the oracle's SpAMM whose leaf products use the
operands rounded to the leaf format (oracle/formats.py, from the format definitions)
and summed in FP64: the only remaining difference is FP32 accumulation, bounded
elementwise by U * 2^-23 * (|A| |B|)_ij + K * 2^-126 with U = K + ceil(K / Kq) + Kq
(parity.tc_bound), K the number of products summed into entry (i, j) (b per
surviving k, three times that for the split forms) and Kq the products of one MMA
instruction (16 for BF16 and FP16, 8 for TF32); the last term covers sums below FP32's
normal range, which the accumulator flushes to zero. The error
against the plain FP64 SpAMM is reported, not asserted beyond a sanity range.
"""
import numpy as np
import pytest

import oracle
from oracle import formats as F
from parity import compare_triples, rel_fro, tc_bound
from paper_1011_3534_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SANITY = {"bf16": 3e-2, "fp16": 3e-3, "tf32": 3e-3, "bf16x3": 1e-4, "tf32x3": 1e-5}
SPLIT = {"bf16x3": "bf16", "tf32x3": "tf32"}


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


def prec_of(S, name):
    return S.PRECISIONS[name]


def gpu_product(S, ctx, A, B, leaf, tau, prec_name, symmetric, sym_product=False, mflags=0):
    n = A.shape[0]
    prec = prec_of(S, prec_name)
    fl = S.COPY_FLAG[prec] | (S.SPAMM_SYMMETRIC if symmetric else 0)
    tA = S.spamm_tree_build(ctx, torch.from_numpy(A).cuda(), n, leaf, fl)
    tB = tA if B is A else S.spamm_tree_build(ctx, torch.from_numpy(B).cuda(), n, leaf, fl)
    tC = S.spamm_multiply(ctx, tA, tB, tau, prec, (S.SPAMM_SYM_PRODUCT if sym_product else 0) | mflags)
    out = dict(C=S.spamm_tree_to_dense(tC), trip=S.spamm_triples(tC), stats=S.spamm_stats(tC),
               norms=[S.spamm_tree_norms(tA, l) for l in range(tA.kmax + 1)])
    S.spamm_tree_free(tC)
    if tB is not tA:
        S.spamm_tree_free(tB)
    S.spamm_tree_free(tA)
    return out


def rounded_operands(X, prec_name):
    if prec_name in SPLIT:
        return F.split(X, SPLIT[prec_name])
    return F.round_to(X, prec_name), None


FP16_MIN_NORMAL = 2.0 ** -14


def reference(A, B, leaf, tau, prec_name, threads):
    """Oracle C with rounded leaf operands and |A||B| over the same triples. For FP16
    also the total magnitude of the products with FP16-subnormal operands, which the
    tensor cores of this GPU do not sum exactly (measured): products of two subnormals
    on the tcgen05 path (leaf 64, 128), products with at least one subnormal operand on
    the warp-level MMA path (leaf 16, 32)."""
    TA, TB = oracle.Tree(A, leaf), oracle.Tree(B, leaf)
    Ah, Al = rounded_operands(A, prec_name)
    Bh, Bl = rounded_operands(B, prec_name)
    T = lambda X: oracle.Tree(X, leaf)
    if prec_name in SPLIT:
        tAh, tAl, tBh, tBl = T(Ah), T(Al), T(Bh), T(Bl)
        Cref = (oracle.spamm_values(TA, TB, tAh, tBh, tau, threads)
                + oracle.spamm_values(TA, TB, tAh, tBl, tau, threads)
                + oracle.spamm_values(TA, TB, tAl, tBh, tau, threads))
        Cabs = oracle.spamm_values(TA, TB, T(np.abs(Ah) + np.abs(Al)), T(np.abs(Bh) + np.abs(Bl)), tau, threads)
    else:
        Cref = oracle.spamm_values(TA, TB, T(Ah), T(Bh), tau, threads)
        Cabs = oracle.spamm_values(TA, TB, T(np.abs(Ah)), T(np.abs(Bh)), tau, threads)
    Csub = 0.0
    if prec_name == "fp16":
        sub = lambda X: np.where(np.abs(X) < FP16_MIN_NORMAL, np.abs(X), 0.0)
        if leaf >= 64:
            Csub = oracle.spamm_values(TA, TB, T(sub(Ah)), T(sub(Bh)), tau, threads)
        else:
            Csub = (oracle.spamm_values(TA, TB, T(sub(Ah)), T(np.abs(Bh)), tau, threads)
                    + oracle.spamm_values(TA, TB, T(np.abs(Ah)), T(sub(Bh)), tau, threads))
    return TA, TB, Cref, Cabs + 0.0, Csub


def check(S, ctx, A, B, leaf, tau, prec_name, symmetric, sym_product=False, mflags=0):
    g = gpu_product(S, ctx, A, B, leaf, tau, prec_name, symmetric, sym_product, mflags)
    thr = oracle.max_threads()
    TA, TB, Cref, Cabs, Csub = reference(A, B, leaf, tau, prec_name, thr)
    ref = oracle.spamm(TA, TB, tau, triples=True, product=False)
    NB = TA.NB
    only_g, only_o = compare_triples(g["trip"], oracle.sort_triples(ref["triples"]), NB,
                                     TA.norm2(TA.kmax), TB.norm2(TB.kmax), tau)
    assert not len(only_g) and not len(only_o), "near-tau flip: rerun with another tau"
    # products summed into each output block
    cnt = np.zeros((NB, NB), dtype=np.int64)
    np.add.at(cnt, (ref["triples"][:, 0], ref["triples"][:, 1]), 1)
    K = leaf * cnt * (3 if prec_name in SPLIT else 1)
    n = A.shape[0]
    Kel = np.repeat(np.repeat(K, leaf, 0), leaf, 1)[:n, :n]
    bound = tc_bound(Kel, prec_name, Cabs) + Csub
    viol = np.abs(g["C"] - Cref) > bound
    assert not np.any(viol), (np.argwhere(viol)[:5], g["C"][viol][:5], Cref[viol][:5])
    C64 = oracle.spamm(TA, TB, tau, threads=thr)["C"]
    err = rel_fro(g["C"], C64)
    print(f"{prec_name} leaf {leaf} n {n} tau {tau}: rel. Frobenius error vs FP64 SpAMM {err:.3e}")
    assert err < SANITY[prec_name]
    st = g["stats"]
    assert st["leaf_products"] + st["mirrored_products"] == ref["count"]
    if tau > 0:   # at tau = 0 the products of absent (padding) leaves survive; the kernel skips them
        assert st["mma_flops"] >= st["leaf_flops"] * (3 if prec_name in SPLIT else 1)
    return g


@pytest.mark.parametrize("prec", ["bf16", "fp16", "tf32", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("n,leaf,tau,kind", [
    (1000, 64, 1e-6, "alg"),      # ragged: 1000 = 15 * 64 + 40
    (2048, 64, 1e-8, "exp"),
    (2100, 128, 1e-6, "alg"),
    (60, 64, 0.0, "exp"),         # one leaf: kmax = 0
])
def test_tc_parity_symmetric(S, ctx, prec, n, leaf, tau, kind):
    A = W.algebraic_decay(n, 2, 0) if kind == "alg" else W.exp_decay(n, 0.85, 1, 0)
    check(S, ctx, A, A, leaf, tau, prec, symmetric=True)


@pytest.mark.parametrize("prec", ["bf16", "fp16", "tf32", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("n,leaf,tau,kind", [
    (1024, 32, 1e-8, "exp"),      # the exp-decay parity workload: n = 1024, 0.85^|i-j|, seed 0
    (1000, 16, 1e-6, "alg"),      # ragged: 1000 = 62 * 16 + 8
    (700, 32, 0.0, "exp"),        # tau = 0: padding blocks survive
    (20, 16, 1e-8, "exp"),        # two leaves, one ragged
])
def test_tc_small_leaves(S, ctx, prec, n, leaf, tau, kind):
    # leaves of 16 and 32 take the warp-level MMA kernel
    A = W.algebraic_decay(n, 2, 0) if kind == "alg" else W.exp_decay(n, 0.85, 1, 0)
    check(S, ctx, A, A, leaf, tau, prec, symmetric=True)


@pytest.mark.parametrize("prec", ["bf16", "tf32", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("leaf", [16, 32, 64, 128])
def test_tc_parity_nonsymmetric(S, ctx, prec, leaf):
    n = 1500
    r = np.random.default_rng(9)
    d = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :])
    A = r.uniform(-1, 1, (n, n)) * 0.9 ** d
    B = np.triu(r.uniform(-1, 1, (n, n)) * 0.93 ** d)
    check(S, ctx, A, B, leaf, 1e-5, prec, symmetric=False)


@pytest.mark.parametrize("prec", ["bf16", "tf32x3", "fp16"])
@pytest.mark.parametrize("n,leaf,tau,kind", [(1000, 64, 1e-6, "alg"), (2100, 128, 1e-6, "alg"), (2048, 64, 1e-8, "exp"),
                                             (60, 64, 0.0, "exp"), (1024, 32, 1e-8, "exp"), (1000, 16, 1e-6, "alg")])
def test_tc_symmetric_product(S, ctx, prec, n, leaf, tau, kind):
    # blocks i <= j multiplied, i > j mirrored: the full triple list, C against the
    # oracle, C symmetric bit for bit; the stored norm trees are symmetric up to the
    # summation order of a block and its transpose
    A = W.algebraic_decay(n, 2, 0) if kind == "alg" else W.exp_decay(n, 0.85, 1, 0)
    g = check(S, ctx, A, A, leaf, tau, prec, symmetric=True, sym_product=True)
    # mirrored blocks are exact transposes; a diagonal block is computed, and is exactly
    # symmetric in the plain formats (the products A_ir A_is are the same numbers),
    # while the split forms sum hi lo and lo hi in separate passes
    C = g["C"]
    blk = np.arange(n) // leaf
    diag = blk[:, None] == blk[None, :]
    asym = np.abs(C - C.T)
    assert not np.any(asym[~diag])
    if prec in SPLIT:
        assert np.all(asym[diag] <= 2.0 ** -20 * np.abs(C).max())
    else:
        assert not np.any(asym[diag])
    for nl in g["norms"]:
        np.testing.assert_allclose(nl, nl.T, rtol=1e-11, atol=0)
    if n > 100:
        assert g["stats"]["mirrored_products"] > 0 and g["stats"]["leaf_products"] < g["stats"]["leaf_products"] + g["stats"]["mirrored_products"]


def test_tc_tau_zero_dense(S, ctx):
    # tau = 0 keeps every triple, including those of padding blocks
    A = W.exp_decay(700, 0.9, 1, 0)
    check(S, ctx, A, A, 64, 0.0, "bf16", symmetric=True)


def test_tc_deterministic(S, ctx):
    A = W.algebraic_decay(3000, 2, 0)
    g1 = gpu_product(S, ctx, A, A, 64, 1e-8, "bf16", True)
    g2 = gpu_product(S, ctx, A, A, 64, 1e-8, "bf16", True)
    assert np.array_equal(g1["C"], g2["C"])


@pytest.mark.parametrize("prec", ["bf16", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("tau", [1e-10, 1e-8, 1e-6, 1e-4])
def test_workload_alg8192_tc_sampled(S, ctx, prec, tau):
    # n = 8192 algebraic decay, leaf 64, in the benchmark's launch configuration:
    # full triple list, C on sampled output blocks against the rounded-operand oracle
    n, leaf = 8192, 64
    A = W.algebraic_decay(n, 2, 0)
    g = gpu_product(S, ctx, A, A, leaf, tau, prec, True, sym_product=True)
    TA = oracle.Tree(A, leaf)
    ref = oracle.spamm(TA, TA, tau, triples=True, product=False)
    compare_triples(g["trip"], oracle.sort_triples(ref["triples"]), TA.NB, TA.norm2(TA.kmax),
                    TA.norm2(TA.kmax), tau)
    Ah, Al = rounded_operands(A, prec)
    tAh = oracle.Tree(Ah, leaf)
    tAl = oracle.Tree(Al, leaf) if Al is not None else None
    tAbs = oracle.Tree(np.abs(Ah) + (np.abs(Al) if Al is not None else 0.0), leaf)
    cnt = np.zeros((TA.NB, TA.NB), dtype=np.int64)
    np.add.at(cnt, (ref["triples"][:, 0], ref["triples"][:, 1]), 1)
    rng = np.random.default_rng(7)
    NB = TA.NB
    blocks = [(0, 0), (0, NB - 1), (NB - 1, NB - 1), (5, 6)] + [tuple(x) for x in rng.integers(0, NB, (12, 2))]
    for i, j in blocks:
        i, j = int(i), int(j)
        if tAl is None:
            Cref = oracle.spamm_block(TA, TA, tau, i, j, tAh, tAh)
        else:
            Cref = (oracle.spamm_block(TA, TA, tau, i, j, tAh, tAh) + oracle.spamm_block(TA, TA, tau, i, j, tAh, tAl)
                    + oracle.spamm_block(TA, TA, tau, i, j, tAl, tAh))
        Cabs = oracle.spamm_block(TA, TA, tau, i, j, tAbs, tAbs)
        K = leaf * cnt[i, j] * (3 if tAl is not None else 1)
        got = g["C"][i * leaf:(i + 1) * leaf, j * leaf:(j + 1) * leaf]
        assert np.all(np.abs(got - Cref) <= tc_bound(K, prec, Cabs)), (i, j)


@pytest.mark.parametrize("n", [4096, 1000, 130])
def test_symmetric_and_transposed_layouts_agree(S, ctx, n):
    # a symmetric operand declared symmetric (one copy serves both roles) and the same
    # operand with transposed copies for the right role: identical norms on and above the
    # diagonal, and identical products from the two operand layouts
    A = W.algebraic_decay(n, 2, 0)
    dA = torch.from_numpy(A).cuda()
    f = S.COPY_FLAG[S.SPAMM_BF16X3]
    t1 = S.spamm_tree_build(ctx, dA, n, 64, f | S.SPAMM_SYMMETRIC)
    t2 = S.spamm_tree_build(ctx, dA, n, 64, f)
    for l in range(t1.kmax + 1):   # on and above the diagonal (a symmetric tree mirrors the rest)
        up = np.triu(np.ones((1 << l, 1 << l), dtype=bool))
        assert np.array_equal(S.spamm_tree_norms(t1, l)[up], S.spamm_tree_norms(t2, l)[up]), l
    c1 = S.spamm_multiply(ctx, t1, t1, 1e-7, S.SPAMM_BF16X3)
    c2 = S.spamm_multiply(ctx, t2, t2, 1e-7, S.SPAMM_BF16X3)
    assert np.array_equal(S.spamm_tree_to_dense(c1), S.spamm_tree_to_dense(c2))
    for t in (c1, c2, t1, t2):
        S.spamm_tree_free(t)


@pytest.mark.parametrize("leaf", [32, 64, 128])
def test_split_tf32_accumulation_bias(S, ctx, leaf):
    # The tensor cores truncate each MMA's FP32 sum; on a product with positive entries a
    # single accumulator per output block gave a mean relative error of -2.2e-5. The split
    # forms keep each pass's hi hi products in an accumulator of their own (leaf 64, 128)
    # or add every MMA's result in FP32 with round to nearest (leaf 32), so the bias
    # against FP64 SpAMM on the same triples is at most that of one pass: leaf / 8 TF32
    # MMAs (K = 8 each), at most half a unit in the last place each on average, hence
    # |mean| <= (leaf / 8) 2^-24 and rms <= (leaf / 8) 2^-23 (the operands' split adds
    # 2^-22 at most)
    n = 2048
    r = np.random.default_rng(17)
    d = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :])
    U = r.uniform(0.5, 1.0, (n, n))
    A = (U + U.T) / 2 * 0.97 ** d          # symmetric, positive, exponential decay
    g = gpu_product(S, ctx, A, A, leaf, 1e-10, "tf32x3", True)
    TA = oracle.Tree(A, leaf)
    C64 = oracle.spamm(TA, TA, 1e-10, threads=oracle.max_threads())["C"]
    big = C64 > 1e-3 * C64.max()
    rel = (g["C"][big] - C64[big]) / C64[big]
    print(f"split TF32 leaf {leaf}: mean relative error {rel.mean():.2e}, rms {np.sqrt((rel ** 2).mean()):.2e}")
    assert abs(rel.mean()) <= (leaf / 8) * 2.0 ** -24
    assert np.sqrt((rel ** 2).mean()) <= (leaf / 8) * 2.0 ** -23 + 2.0 ** -22


@pytest.mark.parametrize("prec", ["bf16", "fp16", "tf32", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("n,tau,kind,symp", [(1000, 1e-6, "alg", False), (2048, 1e-8, "exp", True)])
def test_warp_tiles_leaf64(S, ctx, prec, n, tau, kind, symp):
    # leaf 64 in the warp-tile shape (SPAMM_WARP_TILES: one warp per 64 x 64 output
    # block, the block's surviving k only): the oracle's triples and C within the
    # tensor-core bar; with the symmetric product the blocks i > j are exact transposes
    A = W.algebraic_decay(n, 2, 0) if kind == "alg" else W.exp_decay(n, 0.85, 1, 0)
    g = check(S, ctx, A, A, 64, tau, prec, symmetric=True, sym_product=symp, mflags=S.SPAMM_WARP_TILES)
    # the warp shape issues MMAs for surviving products only: no zero-filled halves
    st = g["stats"]
    assert st["mma_flops"] == st["leaf_flops"] * (3 if prec in SPLIT else 1)
    if symp:
        C = g["C"]
        blk = np.arange(n) // 64
        off = blk[:, None] != blk[None, :]
        assert np.array_equal(C[off], C.T[off])


def test_warp_tiles_flag_checks(S, ctx):
    A = W.exp_decay(512, 0.85, 1, 0)
    t128 = S.spamm_tree_build(ctx, torch.from_numpy(A).cuda(), 512, 128, S.COPY_FLAG[S.SPAMM_BF16] | S.SPAMM_SYMMETRIC)
    with pytest.raises(S.SpammError) as e:
        S.spamm_multiply(ctx, t128, t128, 1e-6, S.SPAMM_BF16, S.SPAMM_WARP_TILES)
    assert e.value.status == S.SPAMM_EUNSUPPORTED
    t64 = S.spamm_tree_build(ctx, torch.from_numpy(A).cuda(), 512, 64, S.SPAMM_KEEP_FP64 | S.SPAMM_SYMMETRIC)
    with pytest.raises(S.SpammError) as e:
        S.spamm_multiply(ctx, t64, t64, 1e-6, S.SPAMM_FP64, S.SPAMM_WARP_TILES)
    assert e.value.status == S.SPAMM_EINVAL
    S.spamm_tree_free(t128)
    S.spamm_tree_free(t64)
