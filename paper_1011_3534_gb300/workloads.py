"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generation only: no step of the SpAMM method (no norms, no
culling, no products). Both the CPU oracle and the CUDA path take their inputs from
here, so the two sides always see the same FP64 buffers.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the t-th
draw of a stream with key s is mix64(s + (t + 1) * 0x9E3779B97F4A7C15), and a
U[0,1) variate is the top 53 bits times 2^-53. A stream key is derived from
(workload id, seed, matrix index, stream id). Symmetric matrices draw element
(i, j) at counter min(i,j) * n + max(i,j), so u_ij = u_ji by construction.

Decay classes follow the paper's definitions of exponential decay
|a_ij| < c * lam^|i-j| and algebraic decay |a_ij| < c / (|i-j|^lam + 1) (Sec. I,
footnote 1), with index separation standing in for physical distance, or a real
distance between lattice sites ordered along a space-filling curve (Sec. II,
Fig. 2; Morton order here).
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_M64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15
_MIX1 = 0xBF58476D1CE4E5B9
_MIX2 = 0x94D049BB133111EB


def _mix64_int(z: int) -> int:
    z &= _M64
    z = ((z ^ (z >> 30)) * _MIX1) & _M64
    z = ((z ^ (z >> 27)) * _MIX2) & _M64
    return z ^ (z >> 31)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = z ^ (z >> np.uint64(30))
        z = z * np.uint64(_MIX1)
        z = z ^ (z >> np.uint64(27))
        z = z * np.uint64(_MIX2)
        z = z ^ (z >> np.uint64(31))
    return z


def stream_key(workload: int, seed: int, matrix: int, stream: int) -> int:
    k = _mix64_int(0x5350414D4D000000 ^ workload)  # "SPAMM" tag
    k = _mix64_int(k ^ seed)
    k = _mix64_int(k ^ matrix)
    k = _mix64_int(k ^ stream)
    return k


def uniform(key: int, counter: np.ndarray) -> np.ndarray:
    """U[0,1) draws of stream `key` at the given uint64 counters."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(key) + (c + np.uint64(1)) * np.uint64(_GAMMA)
    bits = _mix64(state) >> np.uint64(11)
    return bits.astype(np.float64) * (1.0 / 9007199254740992.0)


def _row_chunks(n: int, rows: int = 256):
    return [(r0, min(n, r0 + rows)) for r0 in range(0, n, rows)]


def _parallel_rows(n: int, fill) -> np.ndarray:
    """Fill an n x n FP64 matrix chunk by chunk of rows on host threads."""
    out = np.empty((n, n), dtype=np.float64)
    chunks = _row_chunks(n)
    workers = min(len(chunks), os.cpu_count() or 1, 16)
    if workers <= 1:
        for r0, r1 in chunks:
            fill(out, r0, r1)
    else:
        with ThreadPoolExecutor(workers) as ex:
            list(ex.map(lambda rc: fill(out, rc[0], rc[1]), chunks))
    return out


def _sym_counters(n: int, r0: int, r1: int) -> tuple[np.ndarray, np.ndarray]:
    i = np.arange(r0, r1, dtype=np.int64)[:, None]
    j = np.arange(n, dtype=np.int64)[None, :]
    lo = np.minimum(i, j)
    hi = np.maximum(i, j)
    cnt = (lo * n + hi).astype(np.uint64)
    dist = np.abs(i - j).astype(np.float64)
    return cnt, dist


def exp_decay(n: int, lam: float, workload: int, seed: int, matrix: int = 0) -> np.ndarray:
    """Symmetric a_ij = u_ij * lam^|i-j|, u ~ U[-1, 1] (exponential decay class)."""
    key = stream_key(workload, seed, matrix, 0)

    def fill(out, r0, r1):
        cnt, dist = _sym_counters(n, r0, r1)
        u = 2.0 * uniform(key, cnt) - 1.0
        out[r0:r1] = u * np.power(lam, dist)

    return _parallel_rows(n, fill)


def algebraic_decay(n: int, workload: int, seed: int, matrix: int = 0) -> np.ndarray:
    """Symmetric a_ij = u_ij / (|i-j|^3 + 1), u = U[0.5, 1] * random sign."""
    kmag = stream_key(workload, seed, matrix, 0)
    ksgn = stream_key(workload, seed, matrix, 1)

    def fill(out, r0, r1):
        cnt, dist = _sym_counters(n, r0, r1)
        mag = 0.5 + 0.5 * uniform(kmag, cnt)
        sgn = np.where(uniform(ksgn, cnt) < 0.5, 1.0, -1.0)
        out[r0:r1] = (mag * sgn) / (dist * dist * dist + 1.0)

    return _parallel_rows(n, fill)


def morton3(x: np.ndarray, y: np.ndarray, z: np.ndarray, bits: int) -> np.ndarray:
    """Bit-interleaved (Morton / Z-order) index of integer lattice coordinates."""
    code = np.zeros(np.broadcast(x, y, z).shape, dtype=np.int64)
    for b in range(bits):
        code |= ((np.asarray(x) >> b) & 1).astype(np.int64) << (3 * b)
        code |= ((np.asarray(y) >> b) & 1).astype(np.int64) << (3 * b + 1)
        code |= ((np.asarray(z) >> b) & 1).astype(np.int64) << (3 * b + 2)
    return code


def hilbert3(x: np.ndarray, y: np.ndarray, z: np.ndarray, bits: int) -> np.ndarray:
    """Index of integer lattice coordinates along the 3-D Hilbert curve of 2^bits points
    per side, by Skilling's transform ("Programming the Hilbert curve", AIP Conf. Proc.
    707, 2004): the coordinates are turned into the curve's transposed form (undo the
    excess work of each level, then Gray-code), whose bits, interleaved, are the index."""
    X = [np.asarray(x, dtype=np.int64).copy(), np.asarray(y, dtype=np.int64).copy(),
         np.asarray(z, dtype=np.int64).copy()]
    X = list(np.broadcast_arrays(*X))
    X = [a.copy() for a in X]
    m = 1 << (bits - 1)
    q = m
    while q > 1:                       # inverse undo
        p = q - 1
        for i in range(3):
            hit = (X[i] & q) != 0
            X[0] = np.where(hit, X[0] ^ p, X[0])                 # invert the low bits
            t = np.where(hit, 0, (X[0] ^ X[i]) & p)              # else exchange them
            X[0] ^= t
            X[i] ^= t
        q >>= 1
    for i in range(1, 3):              # Gray encode
        X[i] ^= X[i - 1]
    t = np.zeros_like(X[0])
    q = m
    while q > 1:
        t = np.where((X[2] & q) != 0, t ^ (q - 1), t)
        q >>= 1
    for i in range(3):
        X[i] ^= t
    code = np.zeros_like(X[0])
    for b in range(bits - 1, -1, -1):  # interleave: bit b of X[0], X[1], X[2]
        for i in range(3):
            code = (code << 1) | ((X[i] >> b) & 1)
    return code


def site_permutation(side: int, order: str = "morton") -> np.ndarray:
    """perm[s] = Morton rank of the site that comes s-th in `order` ("morton": the
    identity; "hilbert": the 3-D Hilbert curve over the smallest power-of-two cube
    holding the lattice, restricted to its side^3 sites)."""
    n = side ** 3
    if order == "morton":
        return np.arange(n, dtype=np.int64)
    if order != "hilbert":
        raise ValueError(order)
    bits = max(1, int(math.ceil(math.log2(side))))
    g = np.arange(side)
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    x, y, z = x.ravel(), y.ravel(), z.ravel()
    mrank = np.argsort(np.argsort(morton3(x, y, z, bits), kind="stable"), kind="stable")
    return mrank[np.argsort(hilbert3(x, y, z, bits), kind="stable")]


def permute_csr(indptr, indices, data, perm):
    """(indptr, indices, data) of P H P^T with (P H P^T)[s, t] = H[perm[s], perm[t]]."""
    n = indptr.size - 1
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    rows = np.repeat(np.arange(n), np.diff(indptr))
    r, c = inv[rows], inv[indices]
    o = np.lexsort((c, r))
    r, c, v = r[o], c[o], np.asarray(data)[o]
    ip = np.zeros(n + 1, dtype=np.int64)
    np.add.at(ip, r + 1, 1)
    return np.cumsum(ip), c.astype(np.int64), v


def lattice_sites(side: int, jitter: float, workload: int, seed: int) -> np.ndarray:
    """Site positions of a side^3 cubic lattice (spacing 1), jittered by
    U[-jitter, jitter] per coordinate, listed in Morton order: row s is the site
    whose Morton code is s."""
    bits = max(1, int(math.ceil(math.log2(side))))
    g = np.arange(side)
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    x, y, z = x.ravel(), y.ravel(), z.ravel()
    code = morton3(x, y, z, bits)
    order = np.argsort(code, kind="stable")
    pos = np.stack([x[order], y[order], z[order]], axis=1).astype(np.float64)
    s = np.arange(pos.shape[0], dtype=np.uint64)
    for d in range(3):
        key = stream_key(workload, seed, 0, 10 + d)
        pos[:, d] += jitter * (2.0 * uniform(key, s) - 1.0)
    return pos


def physical_decay(side: int = 16, per_site: int = 8, alpha: float = 1.2,
                   jitter: float = 0.1, workload: int = 3, seed: int = 1, order: str = "morton") -> np.ndarray:
    """Symmetric a_ij = exp(-alpha * r_ij) * u_ij, u ~ N(0, 1) (Box-Muller on two
    uniform streams), r_ij the distance between the sites carrying basis
    functions i and j; `per_site` consecutive basis functions share a site. With
    order="hilbert" the same matrix with its sites renumbered along the Hilbert curve."""
    if order != "morton":
        A = physical_decay(side, per_site, alpha, jitter, workload, seed)
        perm = site_permutation(side, order)
        pb = (perm[:, None] * per_site + np.arange(per_site)[None, :]).ravel()
        return A[np.ix_(pb, pb)]
    pos = lattice_sites(side, jitter, workload, seed)
    n = pos.shape[0] * per_site
    k1 = stream_key(workload, seed, 0, 0)
    k2 = stream_key(workload, seed, 0, 1)
    site = np.arange(n) // per_site

    def fill(out, r0, r1):
        cnt, _ = _sym_counters(n, r0, r1)
        u1 = uniform(k1, cnt)
        u2 = uniform(k2, cnt)
        gauss = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)
        pi = pos[site[r0:r1]][:, None, :]
        pj = pos[site][None, :, :]
        r = np.sqrt(np.sum((pi - pj) ** 2, axis=2))
        out[r0:r1] = np.exp(-alpha * r) * gauss

    return _parallel_rows(n, fill)


def batched_shapes(count: int = 256, lo: int = 512, hi: int = 8192, step: int = 64,
                   lam_lo: float = 0.7, lam_hi: float = 0.95, workload: int = 4,
                   seed: int = 3) -> list[tuple[int, float]]:
    """(n_m, lam_m) of a batch: n log-uniform in [lo, hi] rounded to a multiple of
    `step`, lam ~ U[lam_lo, lam_hi]."""
    m = np.arange(count, dtype=np.uint64)
    un = uniform(stream_key(workload, seed, 0, 20), m)
    ul = uniform(stream_key(workload, seed, 0, 21), m)
    out = []
    for t in range(count):
        n = math.exp(math.log(lo) + float(un[t]) * (math.log(hi) - math.log(lo)))
        n = int(min(hi, max(lo, step * round(n / step))))
        out.append((n, lam_lo + (lam_hi - lam_lo) * float(ul[t])))
    return out


def batched_matrix(m: int, n: int, lam: float, workload: int = 4, seed: int = 3) -> np.ndarray:
    return exp_decay(n, lam, workload, seed, matrix=m)


def tight_binding(side: int, workload: int = 5, seed: int = 2, hop: float = -1.0,
                  onsite: float = 2.0, order: str = "morton"):
    """Cubic tight-binding Hamiltonian on side^3 sites with open boundaries, sites
    in Morton order: nearest-neighbour hopping `hop`, on-site energies
    U[-onsite, onsite]. Returns (indptr, indices, data) of a CSR matrix with
    sorted column indices. With order="hilbert" the same Hamiltonian with its sites
    renumbered along the Hilbert curve."""
    if order != "morton":
        ip, ix, d = tight_binding(side, workload, seed, hop, onsite)
        return permute_csr(ip, ix, d, site_permutation(side, order))
    bits = max(1, int(math.ceil(math.log2(side))))
    g = np.arange(side)
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    x, y, z = x.ravel(), y.ravel(), z.ravel()
    code = morton3(x, y, z, bits)
    rank = np.empty(code.max() + 1, dtype=np.int64)
    order = np.argsort(code, kind="stable")
    rank[code[order]] = np.arange(code.size)
    n = side ** 3
    idx = rank[code]  # matrix index of lattice point (x, y, z)
    eps = onsite * (2.0 * uniform(stream_key(workload, seed, 0, 0), np.arange(n, dtype=np.uint64)) - 1.0)
    rows = [np.arange(n)]
    cols = [np.arange(n)]
    vals = [eps]
    for dx, dy, dz in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
        ok = (x + dx < side) & (y + dy < side) & (z + dz < side)
        a = idx[ok]
        nb_code = morton3(x[ok] + dx, y[ok] + dy, z[ok] + dz, bits)
        b = rank[nb_code]
        rows += [a, b]
        cols += [b, a]
        vals += [np.full(a.size, hop), np.full(a.size, hop)]
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    o = np.lexsort((c, r))
    r, c, v = r[o], c[o], v[o]
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(indptr, r + 1, 1)
    indptr = np.cumsum(indptr)
    return indptr, c.astype(np.int64), v


def csr_to_dense(n: int, indptr, indices, data) -> np.ndarray:
    out = np.zeros((n, n), dtype=np.float64)
    for i in range(n):
        out[i, indices[indptr[i]:indptr[i + 1]]] = data[indptr[i]:indptr[i + 1]]
    return out


def fig1_pair(which: str, n: int = 512) -> tuple[np.ndarray, np.ndarray]:
    """The two synthetic operand pairs of the paper's Fig. 1 (n = 512):
    'A': A_ij = exp(-|i-j|), B_ij = exp(-2|i-j|);
    'B': A_ij = B_ij = 1/|i-j|^3 off the diagonal, 0 on it."""
    d = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :]).astype(np.float64)
    if which == "A":
        return np.exp(-d), np.exp(-2.0 * d)
    if which == "B":
        with np.errstate(divide="ignore"):
            m = np.where(d > 0, 1.0 / (d * d * d), 0.0)
        return m, m.copy()
    raise ValueError(which)


# The configurations of the paper-shaped workloads (sizes, decay law, leaf, tau).
WORKLOADS = {
    "exp1024": dict(n=1024, leaf=32, taus=(1e-8,), make=lambda: exp_decay(1024, 0.85, 1, 0)),
    "alg8192": dict(n=8192, leaf=64, taus=(1e-10, 1e-8, 1e-6, 1e-4),
                    make=lambda: algebraic_decay(8192, 2, 0)),
    "lattice32768": dict(n=32768, leaf=64, taus=(1e-8, 1e-6, 1e-4),
                         make=lambda: physical_decay()),
}
