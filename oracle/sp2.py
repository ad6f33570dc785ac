"""SP2 density-matrix purification oracles: TEST INFRASTRUCTURE ONLY.

The paper applies SpAMM inside the TC2 purification that builds the projector
P = theta[F - mu I] (Sec. III, citing Niklasson's second-order trace-correcting
method): starting from the Hamiltonian mapped onto [0, 1] with occupied states near 1,
each step replaces X by X^2 or by 2X - X^2, whichever moves Tr X towards the electron
count; the energy Tr(H X) measures the accumulated error (Sec. III).

Readings taken here: Gershgorin bounds give the spectral interval,
X0 = (eps_max I - H) / (eps_max - eps_min); the step with t1 = Tr X, t2 = Tr X^2 takes
X^2 when |t2 - N_occ| <= |2 t1 - t2 - N_occ| (ties to X^2), else 2X - X^2; a fixed
number of steps; E = Tr(H X_S) without spin factor.

Two independent implementations:
  sp2_dense    : the loop on dense FP64 matrices (numpy matmul per step);
  sp2_spectral : the same polynomial maps applied to the eigenvalues of H (X commutes
                 with H, so Tr X = sum f(lambda_k) and Tr(H X) = sum eps_k f(lambda_k)).
"""
from __future__ import annotations

import numpy as np


def gershgorin(indptr, indices, data, n: int) -> tuple[float, float]:
    """Gershgorin interval of a symmetric CSR matrix: min/max of H_ii -/+ sum_{j!=i} |H_ij|."""
    lo, hi = np.inf, -np.inf
    for i in range(n):
        cols = indices[indptr[i]:indptr[i + 1]]
        vals = data[indptr[i]:indptr[i + 1]]
        d = float(vals[cols == i].sum())
        r = float(np.abs(vals[cols != i]).sum())
        lo = min(lo, d - r)
        hi = max(hi, d + r)
    return lo, hi


def choose_square(t1: float, t2: float, n_occ: float) -> bool:
    """True: X <- X^2 (the trace-correcting branch rule, ties to X^2)."""
    return abs(t2 - n_occ) <= abs(2.0 * t1 - t2 - n_occ)


def sp2_dense(H: np.ndarray, n_occ: float, steps: int, emin: float, emax: float) -> dict:
    n = H.shape[0]
    X = (emax * np.eye(n) - H) / (emax - emin)
    traces, branches = [float(np.trace(X))], []
    for _ in range(steps):
        X2 = X @ X
        t1, t2 = float(np.trace(X)), float(np.trace(X2))
        sq = choose_square(t1, t2, n_occ)
        X = X2 if sq else 2.0 * X - X2
        branches.append(1 if sq else 0)
        traces.append(float(np.trace(X)))
    return {"energy": float(np.sum(H * X.T)), "traces": traces, "branches": branches, "X": X}


def sp2_spectral(eigs: np.ndarray, n_occ: float, steps: int, emin: float, emax: float) -> dict:
    lam = (emax - np.asarray(eigs, dtype=np.float64)) / (emax - emin)
    traces, branches = [float(lam.sum())], []
    for _ in range(steps):
        t1, t2 = float(lam.sum()), float((lam * lam).sum())
        sq = choose_square(t1, t2, n_occ)
        lam = lam * lam if sq else 2.0 * lam - lam * lam
        branches.append(1 if sq else 0)
        traces.append(float(lam.sum()))
    return {"energy": float(np.dot(eigs, lam)), "traces": traces, "branches": branches}


def spectrum(indptr, indices, data, n: int) -> np.ndarray:
    """Eigenvalues of a symmetric CSR matrix, ascending: the dense FP64 matrix handed to
    LAPACK's symmetric eigensolver (numpy.linalg.eigvalsh). The input of sp2_spectral."""
    H = np.zeros((n, n), dtype=np.float64)
    for i in range(n):
        H[i, indices[indptr[i]:indptr[i + 1]]] = data[indptr[i]:indptr[i + 1]]
    return np.linalg.eigvalsh(H)


def drop_blocks(P: np.ndarray, b: int, tau: float) -> tuple[np.ndarray, int]:
    """The dropping filter of scheme (I) (Sec. III) at b x b resolution: every block of
    the zero-padded P whose Frobenius norm is below tau set to zero. Returns the
    filtered n x n matrix and the number of nonzero blocks kept."""
    n = P.shape[0]
    nb = -(-n // b)
    Q = np.zeros((nb * b, nb * b))
    Q[:n, :n] = P
    blocks = Q.reshape(nb, b, nb, b)
    norm = np.sqrt((blocks ** 2).sum(axis=(1, 3)))
    drop = norm < tau
    blocks[drop[:, None, :, None].repeat(b, 1).repeat(b, 3)] = 0.0
    kept = int(np.count_nonzero(~drop & (norm > 0)))
    return Q[:n, :n].copy(), kept


def block_products(X: np.ndarray, b: int, upper: bool = True) -> int:
    """Leaf products of an exact block-sparse X X: triples (i, j, k) whose blocks X_ik and
    X_kj are both nonzero (only output blocks i <= j when `upper`)."""
    n = X.shape[0]
    nb = -(-n // b)
    Q = np.zeros((nb * b, nb * b))
    Q[:n, :n] = X
    nzb = (np.abs(Q.reshape(nb, b, nb, b)).sum(axis=(1, 3)) > 0).astype(np.int64)
    cnt = nzb @ nzb                       # cnt[i, j] = #k with X_ik, X_kj nonzero
    return int(np.triu(cnt).sum() if upper else cnt.sum())


def sp2_dense_dropping(H: np.ndarray, n_occ: float, steps: int, emin: float, emax: float, b: int,
                       tau: float) -> dict:
    """SP2 by scheme (I) of Sec. III: each step's product X X exact (dense FP64 matmul),
    then filtered by drop_blocks at tau, and the trace-correcting step taken on the
    filtered product. Also the block products each step's exact sparse multiply needs."""
    n = H.shape[0]
    X = (emax * np.eye(n) - H) / (emax - emin)
    traces, branches, products = [float(np.trace(X))], [], []
    for _ in range(steps):
        products.append(block_products(X, b))
        X2, _ = drop_blocks(X @ X, b, tau)
        t1, t2 = float(np.trace(X)), float(np.trace(X2))
        sq = choose_square(t1, t2, n_occ)
        X = X2 if sq else 2.0 * X - X2
        branches.append(1 if sq else 0)
        traces.append(float(np.trace(X)))
    return {"energy": float(np.sum(H * X.T)), "traces": traces, "branches": branches, "X": X,
            "leaf_products": products}
