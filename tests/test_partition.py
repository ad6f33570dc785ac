"""Product-space partition over ranks (paper Sec. II ordering of the product space,
Sec. IV): the planner's segments, the leaves each segment reads, and the one exchange
step, on the host. The exchange runs as world-size-2 gloo ranks on CPU; each rank then
multiplies its output blocks from the leaves it received and the union of the ranks'
blocks is compared with the oracle's product. Not run on GPUs: this pool gives one GPU
per box."""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_1011_3534_gb300 import partition as P
from paper_1011_3534_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def case(n=1000, leaf=64, tau=1e-6):
    A = W.algebraic_decay(n, 2, 0)
    T = oracle.Tree(A, leaf)
    trip = oracle.sort_triples(oracle.spamm(T, T, tau, triples=True, product=False)["triples"])
    return A, T, trip


@pytest.mark.parametrize("curve", ["morton", "hilbert"])
def test_curves_visit_every_block_once(curve):
    bits = 4
    NB = 1 << bits
    ii, jj = np.meshgrid(np.arange(NB), np.arange(NB), indexing="ij")
    f = P.morton2 if curve == "morton" else P.hilbert2
    key = f(ii.ravel(), jj.ravel(), bits)
    assert sorted(key.tolist()) == list(range(NB * NB))
    if curve == "hilbert":   # consecutive cells of the Hilbert curve are neighbours
        order = np.argsort(key)
        di = np.abs(np.diff(ii.ravel()[order])) + np.abs(np.diff(jj.ravel()[order]))
        assert np.all(di == 1)
    else:                    # Z-order keeps every aligned 2^l x 2^l quadrant contiguous
        order = np.argsort(key)
        q = (ii.ravel()[order] // 4) * NB + jj.ravel()[order] // 4
        assert np.all(np.diff(np.flatnonzero(np.diff(q) != 0)) == 16)


@pytest.mark.parametrize("ranks", [1, 2, 3, 8])
@pytest.mark.parametrize("curve", ["morton", "hilbert"])
def test_plan_covers_and_balances(ranks, curve):
    A, T, trip = case()
    w = P.block_work(trip, T.NB, T.leaf, block_cost=2.0 * T.leaf ** 3)
    p = P.plan(w, ranks, curve)
    r = p["rank_of"]
    assert r.min() >= 0 and r.max() <= ranks - 1
    # contiguous along the curve and non-decreasing
    seq = r[p["order"][:, 0], p["order"][:, 1]]
    assert np.all(np.diff(seq) >= 0)
    assert np.isclose(p["loads"].sum(), w.sum())
    # every rank within one block's work of the mean
    assert np.all(np.abs(p["loads"] - w.sum() / ranks) <= w.max() + 1e-9)


def test_needs_are_exactly_the_triples_leaves():
    A, T, trip = case()
    p = P.plan(P.block_work(trip, T.NB, T.leaf), 2)
    na0, nb0 = P.needs(trip, p["rank_of"], 0)
    na1, nb1 = P.needs(trip, p["rank_of"], 1)
    assert na0 | na1 == set(map(tuple, trip[:, [0, 2]].tolist()))
    assert nb0 | nb1 == set(map(tuple, trip[:, [2, 1]].tolist()))


def _tiles(X, leaf, rows):
    n = X.shape[0]
    nb = -(-n // leaf)
    Pd = np.zeros((nb * leaf, nb * leaf))
    Pd[:n, :n] = X
    return {(r, c): Pd[r * leaf:(r + 1) * leaf, c * leaf:(c + 1) * leaf].copy() for r in rows for c in range(nb)}


def _worker(rank, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2")
    dist.init_process_group("gloo", rank=rank, world_size=2)
    n, leaf, tau = 1000, 64, 1e-6
    A, T, trip = case(n, leaf, tau)
    nb = -(-n // leaf)
    p = P.plan(P.block_work(trip, T.NB, leaf), 2)
    need_a, need_b = P.needs(trip, p["rank_of"], rank)
    owner = P.row_owner(nb, 2)
    mine = [r for r in range(nb) if owner[r] == rank]
    got_a, got_b = P.exchange(_tiles(A, leaf, mine), _tiles(A, leaf, mine), need_a, need_b, nb, leaf)
    # the rank's output blocks from its own leaves only, k ascending (Eq. 4 order)
    blocks = {}
    for i, j, k in trip.astype(np.int64).tolist():
        if p["rank_of"][i, j] != rank:
            continue
        blk = blocks.setdefault((i, j), np.zeros((leaf, leaf)))
        blk += got_a[(i, k)] @ got_b[(k, j)]
    out[rank] = dict(blocks=blocks, have_a=sorted(got_a), have_b=sorted(got_b), need_a=sorted(need_a),
                     need_b=sorted(need_b))
    dist.destroy_process_group()


def test_exchange_and_segment_products_gloo():
    import torch.multiprocessing as mp
    port = 28500 + os.getpid() % 1000
    with mp.get_context("spawn").Manager() as m:   # no fork of this (threaded) process
        out = m.dict()
        mp.spawn(_worker, args=(port, out), nprocs=2, join=True)
        res = {r: out[r] for r in (0, 1)}
    n, leaf, tau = 1000, 64, 1e-6
    A, T, trip = case(n, leaf, tau)
    C = oracle.spamm(T, T, tau)["C"]
    nb = -(-n // leaf)
    Cp = np.zeros((nb * leaf, nb * leaf))
    seen = set()
    for r in (0, 1):
        assert res[r]["have_a"] == res[r]["need_a"] and res[r]["have_b"] == res[r]["need_b"]
        for (i, j), blk in res[r]["blocks"].items():
            assert (i, j) not in seen        # each output block on one rank
            seen.add((i, j))
            Cp[i * leaf:(i + 1) * leaf, j * leaf:(j + 1) * leaf] = blk
    assert seen == set(map(tuple, trip[:, :2].tolist()))
    np.testing.assert_allclose(Cp[:n, :n], C, rtol=0, atol=1e-13 * np.abs(C).max())
