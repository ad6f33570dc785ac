"""Product-space partition of one SpAMM product over several ranks (host logic).

The paper proposes to parallelise SpAMM by splitting the product space along a
space-filling curve, weighted by the work that survives the cull, so that every
processor gets a contiguous piece of similar cost (Sec. II, ordering of the product
space; Sec. IV). Output blocks (i, j) are independent once the norm pyramids, a few MB,
are known on every rank, so the split is over output blocks:

  plan()      orders the output leaf blocks along a space-filling curve (Morton or
              Hilbert order of (i, j)), weights each with the work of its surviving
              triples (2 b^3 per leaf product plus a fixed cost per written block), and
              cuts the curve into `ranks` contiguous segments of nearly equal weight.
  needs()     the leaves (i, k) of A and (k, j) of B that a segment's triples read.
  exchange()  one exchange step before compute: every rank starts with the leaf rows it
              owns (a block-row slab of A and of B) and sends each peer the owned leaves
              that peer needs, by point-to-point messages (torch.distributed: NCCL on
              GPUs, gloo on the host); afterwards every rank holds exactly the leaves its
              segment reads and multiplies its output blocks alone.

No rank exchanges partial sums of C (a split over k would add a reduce-scatter; the
output-block split needs none). This module is the partition and exchange logic; the
leaf products of a segment are the single-GPU path's.
"""
from __future__ import annotations

import numpy as np


def morton2(i: np.ndarray, j: np.ndarray, bits: int) -> np.ndarray:
    """Bit-interleaved (Z-order) code of (i, j): bit 2b of the code is bit b of j, bit
    2b + 1 is bit b of i (the quadtree's own order of blocks)."""
    i = np.asarray(i, dtype=np.uint64)
    j = np.asarray(j, dtype=np.uint64)
    code = np.zeros(np.broadcast(i, j).shape, dtype=np.uint64)
    for b in range(bits):
        code |= ((j >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b)
        code |= ((i >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b + 1)
    return code


def hilbert2(i: np.ndarray, j: np.ndarray, bits: int) -> np.ndarray:
    """Index of (i, j) along the 2-D Hilbert curve of side 2^bits (the classic
    rotate-and-flip construction, one quadrant digit per level)."""
    x = np.asarray(j, dtype=np.int64).copy()
    y = np.asarray(i, dtype=np.int64).copy()
    d = np.zeros(np.broadcast(x, y).shape, dtype=np.int64)
    s = 1 << (bits - 1) if bits > 0 else 0
    while s > 0:
        rx = (x & s) > 0
        ry = (y & s) > 0
        d += s * s * ((3 * rx) ^ ry)
        # rotate the quadrant so the sub-curve starts where the parent's piece starts
        flip = ~ry
        swap_x = np.where(flip & rx, s - 1 - x, x)
        swap_y = np.where(flip & rx, s - 1 - y, y)
        x, y = np.where(flip, swap_y, swap_x), np.where(flip, swap_x, swap_y)
        s >>= 1
    return d


def block_work(triples: np.ndarray, nb_padded: int, leaf: int, block_cost: float = 0.0) -> np.ndarray:
    """Work of every output leaf block: 2 leaf^3 per surviving triple (i, j, k), plus
    `block_cost` for each block that has at least one (its epilogue)."""
    w = np.zeros((nb_padded, nb_padded), dtype=np.float64)
    if len(triples):
        np.add.at(w, (triples[:, 0].astype(np.int64), triples[:, 1].astype(np.int64)), 2.0 * leaf ** 3)
    if block_cost:
        w[w > 0] += block_cost
    return w


def plan(work: np.ndarray, ranks: int, curve: str = "morton") -> dict:
    """Contiguous segments of the space-filling curve over the output blocks with
    nearly equal work. Returns dict(order, rank_of, bounds, loads): `order` the blocks
    (i, j) along the curve (blocks without work included, they cost nothing), `rank_of`
    the owning rank of every block (NB x NB), `bounds` the curve positions where each
    rank's segment starts (ranks + 1 entries), `loads` each rank's total work.
    A block goes to the rank whose share [r W / R, (r + 1) W / R) holds the midpoint of
    its work on the running total, so every rank's load is within one block's work of
    W / R."""
    NB = work.shape[0]
    bits = max(0, int(np.ceil(np.log2(NB)))) if NB > 1 else 0
    ii, jj = np.meshgrid(np.arange(NB), np.arange(NB), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    key = morton2(ii, jj, bits) if curve == "morton" else hilbert2(ii, jj, bits)
    order = np.argsort(key, kind="stable")
    w = work.ravel()[order]
    total = float(w.sum())
    mid = np.cumsum(w) - 0.5 * w
    r = np.minimum((mid * ranks / total).astype(np.int64), ranks - 1) if total > 0 else np.zeros(w.size, np.int64)
    r = np.maximum.accumulate(r)              # contiguous and non-decreasing along the curve
    rank_of = np.empty(NB * NB, dtype=np.int64)
    rank_of[order] = r
    bounds = np.searchsorted(r, np.arange(ranks + 1), side="left")
    loads = np.array([w[r == q].sum() for q in range(ranks)])
    return dict(order=np.stack([ii[order], jj[order]], 1), rank_of=rank_of.reshape(NB, NB), bounds=bounds,
                loads=loads)


def needs(triples: np.ndarray, rank_of: np.ndarray, rank: int) -> tuple[set, set]:
    """Leaves (i, k) of A and (k, j) of B read by the triples of `rank`'s output blocks."""
    t = triples.astype(np.int64)
    mine = rank_of[t[:, 0], t[:, 1]] == rank
    t = t[mine]
    return set(map(tuple, t[:, [0, 2]].tolist())), set(map(tuple, t[:, [2, 1]].tolist()))


def row_owner(nb: int, ranks: int) -> np.ndarray:
    """Initial distribution: leaf row r of an operand lives on rank r * ranks // nb
    (contiguous block-row slabs)."""
    return (np.arange(nb) * ranks) // nb


def exchange(local_a: dict, local_b: dict, need_a: set, need_b: set, nb: int, leaf: int, group=None) -> tuple[dict, dict]:
    """The one exchange step. `local_a` / `local_b` map a leaf (r, c) to its b x b tile
    for the leaf rows this rank owns (row_owner); `need_a` / `need_b` are this rank's
    needs(). Every rank tells every peer which of the peer's leaves it needs, then sends
    the requested tiles; returns the leaves this rank needs, complete."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    owner = row_owner(nb, world)
    out_a = {k: v for k, v in local_a.items() if k in need_a}
    out_b = {k: v for k, v in local_b.items() if k in need_b}
    # requests: (operand, r, c) triples this rank needs from each peer
    req = [[] for _ in range(world)]
    for op, need in ((0, need_a), (1, need_b)):
        for (r, c) in sorted(need):
            if owner[r] != rank:
                req[owner[r]].append((op, r, c))
    counts = torch.tensor([len(q) for q in req], dtype=torch.int64)
    all_counts = [torch.zeros(world, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(all_counts, counts, group=group)
    # send my requests to each owner, receive the requests of every peer
    incoming = [None] * world
    ops = []
    for p in range(world):
        if p == rank:
            continue
        if len(req[p]):
            ops.append(dist.isend(torch.tensor(req[p], dtype=torch.int64), p, group=group))
        n_in = int(all_counts[p][rank])
        if n_in:
            incoming[p] = torch.empty((n_in, 3), dtype=torch.int64)
            ops.append(dist.irecv(incoming[p], p, group=group))
    for o in ops:
        o.wait()
    # answer: the requested tiles, in request order, one message per peer
    ops = []
    recv_tiles = {}
    for p in range(world):
        if p == rank:
            continue
        if incoming[p] is not None:
            tiles = [(local_a if op == 0 else local_b)[(r, c)] for op, r, c in incoming[p].tolist()]
            ops.append(dist.isend(torch.from_numpy(np.stack(tiles)), p, group=group))
        if len(req[p]):
            recv_tiles[p] = torch.empty((len(req[p]), leaf, leaf), dtype=torch.float64)
            ops.append(dist.irecv(recv_tiles[p], p, group=group))
    for o in ops:
        o.wait()
    for p, buf in recv_tiles.items():
        for (op, r, c), tile in zip(req[p], buf.numpy()):
            (out_a if op == 0 else out_b)[(r, c)] = tile.copy()
    return out_a, out_b
