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


def system(side, order="morton"):
    ip, ix, d = W.tight_binding(side, order=order)
    n = side ** 3
    H = W.csr_to_dense(n, ip, ix, d)
    lo, hi = O.gershgorin(ip, ix, d, n)
    return (ip, ix, d), H, n, lo, hi


@pytest.mark.parametrize("side,leaf,order", [(8, 16, "morton"), (8, 32, "morton"), (10, 64, "morton"),
                                             (8, 32, "hilbert")])
def test_sp2_fp64_tau0_matches_dense(S, ctx, side, leaf, order):
    (ip, ix, d), H, n, lo, hi = system(side, order)
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


# ---------------------------------------------------------------- scheme (I): dropping

@pytest.mark.parametrize("n,leaf,prec_name", [(1000, 32, "fp64"), (2048, 64, "bf16")])
def test_drop_blocks_matches_oracle_filter(S, ctx, n, leaf, prec_name):
    # the filter keeps exactly the blocks whose norm reaches tau (FP64 tiles: the dense
    # image equals the oracle's filtered matrix bit for bit; BF16 trees keep FP32 tiles
    # of the rounded product, so their presence pattern is compared)
    A = W.algebraic_decay(n, 2, 5)
    prec = S.PRECISIONS[prec_name]
    fl = (S.SPAMM_KEEP_FP64 if prec == S.SPAMM_FP64 else S.COPY_FLAG[prec]) | S.SPAMM_SYMMETRIC
    tA = S.spamm_tree_build(ctx, torch.from_numpy(A).cuda(), n, leaf, fl)
    tC = S.spamm_multiply(ctx, tA, tA, 0.0, prec, S.SPAMM_SYM_PRODUCT)
    C = S.spamm_tree_to_dense(tC)
    nb = -(-n // leaf)
    Q = np.zeros((nb * leaf, nb * leaf))
    Q[:n, :n] = C
    norm = np.sqrt((Q.reshape(nb, leaf, nb, leaf) ** 2).sum(axis=(1, 3)))
    tau = float(np.quantile(norm[norm > 0], 0.6))
    near = np.abs(norm - tau) <= 1e-12 * tau
    kept = S.spamm_drop_blocks(tC, tau)
    Cd = S.spamm_tree_to_dense(tC)
    ref, rkept = O.drop_blocks(C, leaf, tau)
    assert abs(kept - rkept) <= int(near.sum())
    Qd = np.zeros_like(Q)
    Qd[:n, :n] = Cd
    present = np.abs(Qd.reshape(nb, leaf, nb, leaf)).sum(axis=(1, 3)) > 0
    assert np.array_equal(present[~near], (norm >= tau)[~near])
    if prec_name == "fp64" and not near.any():
        assert np.array_equal(Cd, ref)
    # the norm pyramid was rebuilt: the root holds the filtered matrix's norm
    np.testing.assert_allclose(S.spamm_tree_norms(tC, 0)[0, 0], (Cd ** 2).sum(), rtol=1e-12)
    assert S.spamm_drop_blocks(tC, 0.0) == kept
    S.spamm_tree_free(tC)
    S.spamm_tree_free(tA)


@pytest.mark.parametrize("side,leaf,tau", [(8, 32, 1e-4), (10, 64, 1e-3), (12, 64, 1e-6)])
def test_sp2_scheme_one_matches_oracle(S, ctx, side, leaf, tau):
    # scheme (I): exact products filtered at tau; the same branches, traces and energy as
    # the dense oracle of the scheme, and the same block products per step
    (ip, ix, d), H, n, lo, hi = system(side)
    ref = O.sp2_dense_dropping(H, n / 2, 30, lo, hi, leaf, tau)
    g = S.spamm_sp2_dropping(ctx, ip, ix, d, n / 2, 30, leaf, S.SPAMM_FP64, tau)
    assert g["branches"] == ref["branches"]
    np.testing.assert_allclose(g["traces"], ref["traces"], rtol=1e-10)
    assert abs(g["energy"] - ref["energy"]) <= 1e-10 * abs(ref["energy"])
    # block products of the exact sparse multiply (near-ties of the filter aside)
    diff = np.abs(np.array(g["leaf_products"]) - np.array(ref["leaf_products"]))
    assert np.all(diff <= 0.01 * np.array(ref["leaf_products"]))
    dense = O.sp2_dense(H, n / 2, 30, lo, hi)["energy"]
    print(f"scheme (I) {side}^3 leaf {leaf} tau {tau}: error {abs(g['energy'] - dense) / abs(dense):.2e}, "
          f"{sum(g['leaf_products'])} block products ({sum(ref['leaf_products'])} in the oracle)")


def golden_spectral(side):
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sp2_tb_spectral.json")
    rec = json.load(open(path))
    return next(s for s in rec["systems"] if s["side"] == side and s["seed"] == 2)


@pytest.mark.parametrize("prec,tau,tol", [("tf32x3", 1e-6, 1e-6), ("bf16x3", 1e-6, 1e-5)])
def test_sp2_32cubed_against_spectral_reference(S, ctx, prec, tau, tol):
    # 32^3 sites (n = 32768, seed 2), 30 steps, leaf 64: split-precision SpAMM SP2
    # against the spectral SP2 of the dense FP64 eigensolve of H (tests/golden, written
    # by the CPU oracle): the same Gershgorin interval, the same 30 branches, the energy
    # Tr(H X) within the stated relative error and every trace within ten times it
    ref = golden_spectral(32)
    ip, ix, d = W.tight_binding(32, seed=2)[:3]
    n = 32 ** 3
    r = S.spamm_sp2(ctx, ip, ix, d, n / 2, 30, 64, S.PRECISIONS[prec], tau)
    assert abs(r["eps_min"] - ref["emin"]) <= 1e-13 * abs(ref["emin"])
    assert abs(r["eps_max"] - ref["emax"]) <= 1e-13 * abs(ref["emax"])
    assert r["branches"] == ref["branches"]
    np.testing.assert_allclose(r["traces"], ref["traces"], rtol=10 * tol, atol=0)
    err = abs(r["energy"] - ref["energy"]) / abs(ref["energy"])
    print(f"sp2 32^3 {prec} tau {tau}: energy error vs spectral {err:.2e}, {sum(r['leaf_products'])} leaf products, "
          f"{r['ms']:.0f} ms")
    assert err <= tol

