"""GPU parity on the physical-distance decay workload at full size: n = 32768 (4096
sites of a jittered 16^3 lattice in Morton order, 8 basis functions per site,
a_ij = exp(-1.2 r_ij) u_ij, u ~ N(0, 1), seed 1), FP16 and BF16 leaves, leaf 64 and 128,
in the launch configuration of the benchmark's lattice mode.

The oracle finishes the full cull at this size in seconds, so the whole surviving
triple list is compared (bit for bit outside the near-tau band); C is compared on
sampled output blocks (block row 0, diagonal blocks, random blocks from seed 7), each
computed by the oracle one by one with the leaf operands rounded to the leaf format,
within the FP32-accumulation bound of test_gpu_tc.py.
"""
import numpy as np
import pytest

import oracle
from oracle import formats as F
from parity import compare_triples, tc_bound
from paper_1011_3534_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FP16_MIN_NORMAL = 2.0 ** -14


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


@pytest.fixture(scope="module")
def A():
    return W.physical_decay(16, 8, 1.2, 0.1, 3, 1)


@pytest.mark.parametrize("leaf,prec,tau,sym", [(64, "bf16", 1e-6, False), (128, "fp16", 1e-4, False),
                                              (64, "bf16", 1e-6, True), (128, "bf16", 1e-4, True)])
def test_lattice32768_parity(S, ctx, A, leaf, prec, tau, sym):
    # sym: the benchmark's lattice mode, a symmetric operand with the symmetric product
    # (blocks i <= j multiplied, C_ji = C_ij^T written by the epilogue)
    n = A.shape[0]
    assert n == 32768
    p = S.PRECISIONS[prec]
    fl = S.COPY_FLAG[p] | S.SPAMM_SYMMETRIC | (S.SPAMM_NO_RIGHT if sym else 0)
    tA = S.spamm_tree_build(ctx, torch.from_numpy(A).cuda(), n, leaf, fl)
    tC = S.spamm_multiply(ctx, tA, tA, tau, p, S.SPAMM_SYM_PRODUCT if sym else 0)
    trip = S.spamm_triples(tC)
    st = S.spamm_stats(tC)
    TA = oracle.Tree(A, leaf)
    ref = oracle.spamm(TA, TA, tau, triples=True, product=False, threads=oracle.max_threads())
    NB = TA.NB
    only_g, only_o = compare_triples(trip, oracle.sort_triples(ref["triples"]), NB, TA.norm2(TA.kmax),
                                     TA.norm2(TA.kmax), tau)
    assert st["leaf_products"] + st["mirrored_products"] == ref["count"] + len(only_g) - len(only_o)
    print(f"lattice n={n} leaf {leaf} {prec} tau {tau}: {ref['count']} surviving triples of {NB ** 3}")
    # sampled output blocks against the rounded-operand oracle
    Ar = F.round_to(A, prec)
    tAr = oracle.Tree(Ar, leaf)
    tAbs = oracle.Tree(np.abs(Ar), leaf)
    sub = oracle.Tree(np.where(np.abs(Ar) < FP16_MIN_NORMAL, np.abs(Ar), 0.0), leaf) if prec == "fp16" else None
    cnt = np.zeros((NB, NB), dtype=np.int64)
    np.add.at(cnt, (ref["triples"][:, 0], ref["triples"][:, 1]), 1)
    nb = -(-n // leaf)
    rng = np.random.default_rng(7)
    blocks = [(0, j) for j in range(0, nb, max(1, nb // 8))] + [(i, i) for i in range(0, nb, max(1, nb // 8))]
    blocks += [tuple(int(v) for v in x) for x in rng.integers(0, nb, (12, 2))]
    blocks += [(j, i) for i, j in blocks if i != j][:8]   # mirrored blocks of a symmetric product
    C = S.spamm_tree_to_dense(tC)
    for i, j in blocks:
        Cref = oracle.spamm_block(TA, TA, tau, i, j, tAr, tAr)
        Cabs = oracle.spamm_block(TA, TA, tau, i, j, tAbs, tAbs)
        Csub = oracle.spamm_block(TA, TA, tau, i, j, sub, sub) if sub is not None else 0.0
        K = leaf * cnt[i, j]
        got = C[i * leaf:(i + 1) * leaf, j * leaf:(j + 1) * leaf]
        bad = np.abs(got - Cref) > tc_bound(K, prec, Cabs) + Csub
        assert not np.any(bad), (i, j, np.argwhere(bad)[:3])
    S.spamm_tree_free(tC)
    S.spamm_tree_free(tA)
