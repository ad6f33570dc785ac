"""SP2 purification on SpAMM products (GPU) against the dense FP64 SP2 oracle.

At tau = 0 the FP64 SpAMM products are exact up to rounding, so the energy, the
traces and the branch sequence must match the dense oracle (energy within 1e-12
relative). Tensor-core precisions and tau > 0 are compared at stated tolerances.
"""
import numpy as np
import pytest

from oracle import sp2 as O
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


def system(side):
    ip, ix, d = W.tight_binding(side)
    n = side ** 3
    H = W.csr_to_dense(n, ip, ix, d)
    lo, hi = O.gershgorin(ip, ix, d, n)
    return (ip, ix, d), H, n, lo, hi


@pytest.mark.parametrize("side,leaf", [(8, 16), (8, 32), (10, 64)])
def test_sp2_fp64_tau0_matches_dense(S, ctx, side, leaf):
    (ip, ix, d), H, n, lo, hi = system(side)
    ref = O.sp2_dense(H, n / 2, 30, lo, hi)
    g = S.spamm_sp2(ctx, ip, ix, d, n / 2, 30, leaf, S.SPAMM_FP64, 0.0)
    assert g["eps_min"] == pytest.approx(lo, rel=1e-15) and g["eps_max"] == pytest.approx(hi, rel=1e-15)
    assert g["branches"] == ref["branches"]
    np.testing.assert_allclose(g["traces"], ref["traces"], rtol=1e-11)
    assert abs(g["energy"] - ref["energy"]) <= 1e-12 * abs(ref["energy"])
    nb = -(-n // leaf)
    NB = 1 << (nb - 1).bit_length()
    assert all(lp == NB ** 3 for lp in g["leaf_products"])   # tau = 0 keeps every triple


@pytest.mark.parametrize("prec,tol", [("bf16x3", 1e-5), ("tf32", 1e-3), ("bf16", 1e-2)])
def test_sp2_tensor_core_energy(S, ctx, prec, tol):
    (ip, ix, d), H, n, lo, hi = system(10)
    ref = O.sp2_dense(H, n / 2, 30, lo, hi)
    g = S.spamm_sp2(ctx, ip, ix, d, n / 2, 30, 64, S.PRECISIONS[prec], 0.0)
    err = abs(g["energy"] - ref["energy"]) / abs(ref["energy"])
    print(f"SP2 {prec} tau=0 n={n}: relative energy error {err:.3e}, branches equal: {g['branches'] == ref['branches']}")
    assert err < tol


def test_sp2_tau_positive_and_spectral_oracle(S, ctx):
    # n = 4096 (16^3 sites): the dense oracle equals the spectral one; SpAMM at tau > 0
    # skips products and stays close in energy
    (ip, ix, d), H, n, lo, hi = system(16)
    spec = O.sp2_spectral(np.linalg.eigvalsh(H), n / 2, 30, lo, hi)
    g0 = S.spamm_sp2(ctx, ip, ix, d, n / 2, 30, 64, S.SPAMM_FP64, 0.0)
    assert abs(g0["energy"] - spec["energy"]) <= 1e-10 * abs(spec["energy"])
    for tau in (1e-10, 1e-8, 1e-6):
        g = S.spamm_sp2(ctx, ip, ix, d, n / 2, 30, 64, S.SPAMM_FP64, tau)
        err = abs(g["energy"] - spec["energy"]) / abs(spec["energy"])
        print(f"SP2 fp64 tau={tau:g}: relative energy error {err:.3e}, leaf products {sum(g['leaf_products'])}")
        assert err < 1e3 * tau
        assert sum(g["leaf_products"]) < sum(g0["leaf_products"])
