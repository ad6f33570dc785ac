"""Pins of the SP2 purification oracles (CPU)."""
import numpy as np
import pytest

from oracle import sp2 as O
from paper_1011_3534_gb300 import workloads as W


def tb_dense(side):
    ip, ix, d = W.tight_binding(side)
    n = side ** 3
    return W.csr_to_dense(n, ip, ix, d), (ip, ix, d), n


def test_gershgorin_matches_dense_bound():
    H, (ip, ix, d), n = tb_dense(4)
    lo, hi = O.gershgorin(ip, ix, d, n)
    diag = np.diag(H)
    rad = np.abs(H).sum(1) - np.abs(diag)
    assert lo == pytest.approx((diag - rad).min()) and hi == pytest.approx((diag + rad).max())
    ev = np.linalg.eigvalsh(H)
    assert lo <= ev.min() and ev.max() <= hi


@pytest.mark.parametrize("side", [4, 6, 8])
def test_dense_equals_spectral(side):
    H, (ip, ix, d), n = tb_dense(side)
    lo, hi = O.gershgorin(ip, ix, d, n)
    dn = O.sp2_dense(H, n / 2, 30, lo, hi)
    sp = O.sp2_spectral(np.linalg.eigvalsh(H), n / 2, 30, lo, hi)
    assert dn["branches"] == sp["branches"]
    np.testing.assert_allclose(dn["traces"], sp["traces"], rtol=1e-9)
    assert abs(dn["energy"] - sp["energy"]) <= 1e-9 * abs(sp["energy"])


def test_gapped_spectrum_converges_to_projector():
    # a diagonal H with a gap: SP2 drives the occupied eigenvalues to 1 and the rest to
    # 0, so Tr X = N_occ and the energy is the sum of the N_occ lowest levels
    eps = np.concatenate([np.linspace(-2, -1, 50), np.linspace(1, 2, 50)])
    H = np.diag(eps)
    r = O.sp2_dense(H, 50, 40, -2.0, 2.0)
    assert abs(r["traces"][-1] - 50) < 1e-12
    assert abs(r["energy"] - eps[:50].sum()) < 1e-10
    X = r["X"]
    assert np.abs(X @ X - X).max() < 1e-12


def test_hand_worked_two_level():
    # H = diag(-1, 1), N_occ = 1, interval [-1, 1]: X0 = diag(1, 0) is already the
    # projector; Tr X0 = 1, Tr X0^2 = 1 -> |1 - 1| <= |2 - 1 - 1| ties to X^2, and the
    # iterate never changes; E = -1
    r = O.sp2_dense(np.diag([-1.0, 1.0]), 1.0, 5, -1.0, 1.0)
    assert r["branches"] == [1] * 5 and r["energy"] == -1.0
    # X0 = diag(0.75, 0.25) (interval [-2, 2]): t1 = 1, t2 = 0.625; |0.625 - 1| = 0.375
    # vs |2 - 0.625 - 1| = 0.375: tie -> X^2 = diag(0.5625, 0.0625)
    r = O.sp2_dense(np.diag([-1.0, 1.0]), 1.0, 1, -2.0, 2.0)
    assert r["branches"] == [1] and r["traces"][1] == 0.625


def test_traces_stay_in_range():
    H, (ip, ix, d), n = tb_dense(6)
    lo, hi = O.gershgorin(ip, ix, d, n)
    r = O.sp2_spectral(np.linalg.eigvalsh(H), n / 2, 30, lo, hi)
    assert all(0 <= t <= n for t in r["traces"])
    assert abs(r["traces"][-1] - n / 2) < abs(r["traces"][0] - n / 2) + 1e-9


# ---------------------------------------------------------------- scheme (I): dropping

def test_drop_blocks_closed_form():
    # constant blocks c_IJ of side b have Frobenius norm |c_IJ| b: the filter keeps
    # exactly the blocks with |c_IJ| b >= tau, on a ragged order (padding never counts)
    b, nb = 4, 5
    c = np.arange(1, nb * nb + 1, dtype=np.float64).reshape(nb, nb) / 10.0
    P = np.kron(c, np.ones((b, b)))[:18, :18]       # 18 = 4 * 4 + 2: ragged last blocks
    tau = 1.05 * b
    Q, kept = O.drop_blocks(P, b, tau)
    norms = np.zeros((nb, nb))
    for I in range(nb):
        for J in range(nb):
            blk = P[I * b:(I + 1) * b, J * b:(J + 1) * b]
            norms[I, J] = np.sqrt((blk ** 2).sum())
            want = blk if norms[I, J] >= tau else 0.0 * blk
            assert np.array_equal(Q[I * b:(I + 1) * b, J * b:(J + 1) * b], want)
    assert kept == int((norms >= tau).sum())
    # tau = 0 drops nothing; the filter is idempotent
    assert np.array_equal(O.drop_blocks(P, b, 0.0)[0], P)
    assert np.array_equal(O.drop_blocks(Q, b, tau)[0], Q)


def test_block_products_brute_force():
    r = np.random.default_rng(4)
    b, nb = 3, 6
    mask = r.random((nb, nb)) < 0.4
    X = np.kron(mask.astype(float), np.ones((b, b))) * r.uniform(0.5, 1, (nb * b, nb * b))
    want = sum(1 for i in range(nb) for j in range(i, nb) for k in range(nb) if mask[i, k] and mask[k, j])
    assert O.block_products(X, b) == want
    assert O.block_products(X, b, upper=False) == int((mask.astype(int) @ mask.astype(int)).sum())


@pytest.mark.parametrize("side", [4, 6])
def test_dropping_at_zero_is_dense_sp2(side):
    # scheme (I) with tau = 0 drops nothing: the same loop as sp2_dense, bit for bit
    H, (ip, ix, d), n = tb_dense(side)
    lo, hi = O.gershgorin(ip, ix, d, n)
    a = O.sp2_dense(H, n / 2, 20, lo, hi)
    z = O.sp2_dense_dropping(H, n / 2, 20, lo, hi, 8, 0.0)
    assert a["branches"] == z["branches"] and a["traces"] == z["traces"] and a["energy"] == z["energy"]
    assert np.array_equal(a["X"], z["X"])


def test_dropping_error_shrinks_with_tau():
    # the dropped mass goes to zero with tau: the energy error of scheme (I) against
    # dense SP2 falls, and every run keeps no more blocks than the run below it
    H, (ip, ix, d), n = tb_dense(6)
    lo, hi = O.gershgorin(ip, ix, d, n)
    ref = O.sp2_dense(H, n / 2, 25, lo, hi)["energy"]
    errs, prods = [], []
    for tau in (1e-2, 1e-4, 1e-6):
        r = O.sp2_dense_dropping(H, n / 2, 25, lo, hi, 8, tau)
        errs.append(abs(r["energy"] - ref) / abs(ref))
        prods.append(sum(r["leaf_products"]))
    assert errs[2] < errs[0] and errs[2] < 1e-5
    assert prods[0] <= prods[1] <= prods[2]


def _golden_systems():
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sp2_tb_spectral.json")
    return json.load(open(path))["systems"]


@pytest.mark.parametrize("side", [16, 32])
def test_spectral_golden_invariants(side):
    # the stored spectral SP2 references (tests/golden/make_sp2_reference.py) against
    # facts that do not need the eigensolve: the Gershgorin interval of H, the sum of the
    # eigenvalues = Tr H (the sum of the on-site energies), Tr X0 = (n emax - Tr H) /
    # (emax - emin), traces inside [0, n], and 30 branches
    from paper_1011_3534_gb300 import workloads as W
    rec = next(s for s in _golden_systems() if s["side"] == side)
    ip, ix, d = W.tight_binding(side, seed=rec["seed"])[:3]
    n = side ** 3
    lo, hi = O.gershgorin(ip, ix, d, n)
    assert (lo, hi) == (rec["emin"], rec["emax"])
    diag = np.array([d[ip[i]:ip[i + 1]][ix[ip[i]:ip[i + 1]] == i].sum() for i in range(n)])
    trH = float(diag.sum())
    assert abs(rec["eig_sum"] - trH) <= 1e-9 * n
    assert abs(rec["traces"][0] - (n * hi - trH) / (hi - lo)) <= 1e-9 * n
    assert len(rec["branches"]) == 30 and len(rec["traces"]) == 31
    assert all(0.0 <= t <= n for t in rec["traces"])
    assert lo <= rec["eig_min"] and rec["eig_max"] <= hi


def test_spectral_golden_16_equals_the_dense_oracle_run_on_its_spectrum():
    # the 16^3 record is what the spectral oracle gives on the dense eigensolve now
    from paper_1011_3534_gb300 import workloads as W
    rec = next(s for s in _golden_systems() if s["side"] == 16)
    ip, ix, d = W.tight_binding(16, seed=rec["seed"])[:3]
    n = 16 ** 3
    r = O.sp2_spectral(O.spectrum(ip, ix, d, n), n / 2, 30, rec["emin"], rec["emax"])
    assert r["branches"] == rec["branches"]
    assert abs(r["energy"] - rec["energy"]) <= 1e-10 * abs(rec["energy"])
