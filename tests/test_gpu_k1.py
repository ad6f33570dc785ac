"""GPU parity of the leaf-block kernel (K1: Frobenius norms and leaf copies, Eq. 1 and
Sec. III) against the CPU oracle, element by element, through the C ABI.

Leaf copies are compared value for value with oracle/formats.py (round to nearest
even from the format definitions; the split pair hi = fmt(a), lo = fmt(a - hi)): the
copies decide the tensor-core operands, and an error of one unit in the last place of
a low part lies far inside the FP32 bound of the product tests, so only this test can
see it. Norms of every leaf are compared with the oracle's FP64 sums within 1e-13
relative on inputs built to stress the double-float accumulation: elements spanning
many binades inside one round of eight and from one round to the next, zeros, FP64
subnormals, and values at and next to the rounding ties of every format.
"""
import numpy as np
import pytest

import oracle
from oracle import formats as F
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


def adversarial(n, seed, span=80, sym=False):
    """Seeded n x n FP64 input: normal values scaled by 2^U[-span, span] per element, with
    planted zeros, FP64 subnormals, values near 2^-80 and 2^-130 (outside the fast split
    and FP32-normal ranges), exact format values (split low part zero) and exact ties
    and near-ties at the BF16 and TF32/FP16 rounding positions."""
    r = np.random.default_rng(seed)
    X = r.standard_normal((n, n)) * np.exp2(r.uniform(-span, span, (n, n)))
    u = X.view(np.uint64)
    kind = r.integers(0, 16, (n, n))
    one = np.uint64(1)
    tie_bf16 = (u & ~np.uint64((1 << 45) - 1)) | (one << np.uint64(44))   # exactly half a BF16 ulp
    tie_tf32 = (u & ~np.uint64((1 << 42) - 1)) | (one << np.uint64(41))   # exactly half a TF32/FP16 ulp
    u[:] = np.where(kind == 1, tie_bf16, u)
    u[:] = np.where(kind == 2, tie_tf32, u)
    u[:] = np.where(kind == 3, tie_bf16 | one, u)                          # just above the tie
    u[:] = np.where(kind == 4, tie_tf32 - one, u)                          # just below the tie
    u[:] = np.where(kind == 5, u & ~np.uint64((1 << 45) - 1), u)           # exact BF16 value
    u[:] = np.where(kind == 6, u & ~np.uint64((1 << 42) - 1), u)           # exact TF32 value
    X[kind == 7] = 0.0
    X[kind == 8] = r.choice([5e-324, -2.5e-320, 1e-310], size=int((kind == 8).sum()))
    X[kind == 9] = r.standard_normal(int((kind == 9).sum())) * 2.0 ** -80
    X[kind == 10] = r.standard_normal(int((kind == 10).sum())) * 2.0 ** -130
    if sym:
        X = np.triu(X) + np.triu(X, 1).T
    return np.ascontiguousarray(X)


def tiles(X, leaf):
    """X zero-padded to whole leaves, as (nb, nb, leaf, leaf)."""
    n = X.shape[0]
    nb = -(-n // leaf)
    P = np.zeros((nb * leaf, nb * leaf), dtype=X.dtype)
    P[:n, :n] = X
    return P.reshape(nb, leaf, nb, leaf).transpose(0, 2, 1, 3)


def f32_bits(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def bf16_bits(x):
    return (f32_bits(x).view(np.uint32) >> 16).astype(np.uint16)


def fp16_bits(x):
    return np.asarray(x, dtype=np.float64).astype(np.float16).view(np.uint16)


def check_copies(S, t, X, leaf, copies, transposed=False):
    T = tiles(X, leaf)
    if transposed:
        T = T.transpose(0, 1, 3, 2)
    suf = "_t" if transposed else ""
    for name in copies:
        g = S.spamm_tree_leaf_copy(t, name + suf)
        if name in ("tf32", "bf16", "fp16"):
            ref = F.round_to(T, name)
        elif name == "tf32lo":
            ref = F.split(T, "tf32")[1]
        elif name == "bf16lo":
            ref = F.split(T, "bf16")[1]
        elif name == "f64":
            ref = T
        else:
            raise ValueError(name)
        if name in ("bf16", "bf16lo"):
            gv = (g.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        elif name == "fp16":
            gv = g.view(np.float16).astype(np.float64)
            keep = np.abs(T) < 65504.0                # the oracle's rounding does not overflow
            gv, ref = gv[keep], ref[keep]
        else:
            gv = g.astype(np.float64)
        bad = gv != ref
        assert not np.any(bad), (name + suf, np.argwhere(bad)[:5], gv[bad][:5], ref[bad][:5])


COPY_SETS = {"tf32x3": ("tf32", "tf32lo"), "bf16x3": ("bf16", "bf16lo"), "bf16": ("bf16",),
             "tf32": ("tf32",), "fp16": ("fp16",)}


@pytest.mark.parametrize("leaf", [16, 32, 64, 128])
@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "fp16"])
def test_leaf_copies_adversarial(S, ctx, leaf, prec):
    # ragged n (edge leaves padded); FP16 with a narrower span keeps most values in range
    n = 3 * leaf + 5
    X = adversarial(n, 11 + leaf, span=20 if prec == "fp16" else 80)
    p = S.PRECISIONS[prec]
    t = S.spamm_tree_build(ctx, torch.from_numpy(X).cuda(), n, leaf, S.COPY_FLAG[p])
    check_copies(S, t, X, leaf, COPY_SETS[prec])
    check_copies(S, t, X, leaf, COPY_SETS[prec], transposed=True)
    S.spamm_tree_free(t)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_leaf_copies_symmetric_fast_kernels(S, ctx, prec):
    # the specialised copy-set instances (symmetric operand, one orientation, leaf 64
    # and 128, 16-byte loads) on an adversarial symmetric input
    for leaf in (64, 128):
        n = 4 * leaf
        X = adversarial(n, 5 + leaf, sym=True)
        p = S.PRECISIONS[prec]
        t = S.spamm_tree_build(ctx, torch.from_numpy(X).cuda(), n, leaf,
                               S.COPY_FLAG[p] | S.SPAMM_SYMMETRIC | S.SPAMM_NO_RIGHT)
        check_copies(S, t, X, leaf, COPY_SETS[prec])
        S.spamm_tree_free(t)


@pytest.mark.parametrize("leaf", [16, 32, 64, 128])
@pytest.mark.parametrize("span", [20, 80, 200])
def test_leaf_norms_adversarial(S, ctx, leaf, span):
    # every leaf's squared norm within 1e-13 of the oracle's FP64 sum; the elements of a
    # round of eight span up to 2^(2 span) in magnitude, and so do neighbouring rounds
    n = 3 * leaf + 7
    X = adversarial(n, 100 + span + leaf, span=span)
    for flags, sym in ((S.COPY_FLAG[S.SPAMM_TF32X3], False),
                       (S.COPY_FLAG[S.SPAMM_BF16] | S.SPAMM_SYMMETRIC | S.SPAMM_NO_RIGHT, True)):
        Y = adversarial(n, 100 + span + leaf, span=span, sym=True) if sym else X
        t = S.spamm_tree_build(ctx, torch.from_numpy(Y).cuda(), n, leaf, flags)
        g = S.spamm_tree_norms(t, t.kmax)
        ref = oracle.Tree(Y, leaf).norm2(t.kmax)
        rel = np.abs(g - ref) / np.where(ref > 0, ref, 1.0)
        assert np.all((ref > 0) | (g == 0)), "a zero leaf got a nonzero norm"
        assert rel.max() <= 1e-13, (rel.max(), np.unravel_index(rel.argmax(), rel.shape))
        S.spamm_tree_free(t)


def test_headline_split_copies_full_size(S, ctx):
    # the benchmark's input and launch configuration (n = 8192 algebraic decay, leaf 64,
    # symmetric operand, split TF32 and split BF16 copies): every element of both copies
    A = W.algebraic_decay(8192, 2, 0)
    dA = torch.from_numpy(A).cuda()
    for prec in ("tf32x3", "bf16x3"):
        p = S.PRECISIONS[prec]
        t = S.spamm_tree_build(ctx, dA, 8192, 64, S.COPY_FLAG[p] | S.SPAMM_SYMMETRIC | S.SPAMM_NO_RIGHT)
        check_copies(S, t, A, 64, COPY_SETS[prec])
        S.spamm_tree_free(t)
