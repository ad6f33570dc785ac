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
    # tau = 0 keeps every triple; the symmetric products multiply the blocks i <= j
    assert all(lp == NB * NB * (NB + 1) // 2 for lp in g["leaf_products"])


@pytest.mark.parametrize("prec,tol", [("tf32x3", 1e-6), ("bf16x3", 1e-5), ("tf32", 1e-3), ("bf16", 1e-2)])
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


def test_sp2_stepwise_run_equals_one_shot(S, ctx):
    # the run object queues the same kernels in the same order: identical results
    (ip, ix, d), H, n, lo, hi = system(10)
    taus = [1e-9 * (1 + (k % 3)) for k in range(25)]
    one = S.spamm_sp2(ctx, ip, ix, d, n / 2, 25, 64, S.SPAMM_TF32X3, np.array(taus))
    run = S.Sp2Run(ctx, ip, ix, d, n / 2, 64, S.SPAMM_TF32X3)
    for k, t in enumerate(taus):
        run.step(t)
        X = run.iterate()
        assert X.n == n and X.leaf == 64
    two = run.end()
    assert two["energy"] == one["energy"] and two["traces"] == one["traces"]
    assert two["branches"] == one["branches"] and two["leaf_products"] == one["leaf_products"]
    assert two["taus"] == taus


def test_sp2_learned_with_constant_network_equals_fixed_tau(S, ctx):
    # a network predicting log10 error -7 everywhere: with budget 1e-6 every step takes
    # tau_max, with budget 1e-8 every step tau_min; each must equal the fixed-tau loop
    (ip, ix, d), H, n, lo, hi = system(10)
    m = S.Mlp(ctx, S.MLP_FEATURES, 8, seed=0)
    z = np.zeros(m.P, dtype=np.float32)
    z[-1] = -7.0
    m.set_params(z)
    for budget, tau in ((1e-6, 1e-5), (1e-8, 1e-9)):
        g = S.spamm_sp2_learned(ctx, ip, ix, d, n / 2, 20, 64, S.SPAMM_BF16X3, m, budget, 1e-9, 1e-5)
        f = S.spamm_sp2(ctx, ip, ix, d, n / 2, 20, 64, S.SPAMM_BF16X3, tau)
        assert all(abs(t / tau - 1) < 1e-12 for t in g["taus"])
        assert g["energy"] == f["energy"] and g["branches"] == f["branches"]
        assert g["leaf_products"] == f["leaf_products"]
    m.free()
