"""Learned tolerance controller for SpAMM inside SP2 (not in the paper; the paper fixes
tau by hand, Sec. III).

Workflow, all on the GPU through the C ABI:
  collect()   runs the SP2 loop with FP64 products at a fixed tolerance and, at every
              step, labels the product X X at each tau of a grid with the relative
              Frobenius error of the FP64 SpAMM product against the product at tau = 0:
              label = log10(||C_tau - C_0||_F / ||C_0||_F); the features are the
              library's (spamm_features).
  train()     fits the library's network (spamm_mlp_*) to (features, label) pairs.
  conservative_tau()  the largest tau of a half-decade grid whose plain FP64 SP2 energy
              meets a relative error target: the controller's fallback and arbiter.
  calibrate_budget()  the largest per-product error budget of a half-decade grid whose
              learned-tau SP2 energy meets the target on a training system, divided by
              a safety margin (default one decade): near-tie branch decisions of the
              trace-correcting step make the energy error jump when a product error
              crosses a system-dependent threshold, so a budget that just passes on one
              system need not pass on another.
  calibrate_margin()  the same for the branch-margin rule (spamm_sp2_learned_margin): the
              per-product budget is loosened at steps whose trace-correcting decision is
              far from a tie; the settings with the fewest leaf products that meet the
              target with a safety factor on the training system.
"""
from __future__ import annotations

import numpy as np

from . import spamm as S

LABEL_FLOOR = -12.0   # labels below carry no information for budgets of interest


def half_decades(lo: float, hi: float) -> list[float]:
    k0, k1 = int(round(2 * np.log10(lo))), int(round(2 * np.log10(hi)))
    return [10.0 ** (k / 2) for k in range(k0, k1 + 1)]


def collect(ctx, indptr, indices, data, n_occ: float, steps: int, leaf: int, taus, tau_run: float = 0.0):
    """(features [steps * len(taus), 69], labels) along the FP64 SP2 trajectory."""
    run = S.Sp2Run(ctx, indptr, indices, data, n_occ, leaf, S.SPAMM_FP64)
    feats, labels = [], []
    C0 = Ct = None
    try:
        for _ in range(steps):
            X = run.iterate()
            C0 = S.spamm_multiply(ctx, X, X, 0.0, S.SPAMM_FP64, 0, C0)
            for tau in taus:
                Ct = S.spamm_multiply(ctx, X, X, tau, S.SPAMM_FP64, 0, Ct)
                d, r = S.spamm_tree_distance(Ct, C0)
                labels.append(np.log10(d / r) if d > 0 and r > 0 else LABEL_FLOOR)
                feats.append(S.spamm_features(X, X, tau))
            run.step(tau_run)
    finally:
        for t in (C0, Ct):
            if t is not None:
                S.spamm_tree_free(t)
        run.end()
    y = np.maximum(np.asarray(labels, dtype=np.float32), LABEL_FLOOR)
    return np.stack(feats).astype(np.float32), y


def train(ctx, X, y, hidden: int = 32, epochs: int = 300, batch: int = 64, lr: float = 3e-3, seed: int = 0):
    m = S.Mlp(ctx, X.shape[1], hidden, seed=seed)
    loss = m.train(X, y, epochs=epochs, batch=batch, lr=lr, seed=seed + 1)
    return m, loss


def energy_error(res: dict, e_ref: float) -> float:
    return abs(res["energy"] - e_ref) / abs(e_ref)


def conservative_tau(ctx, csr, n_occ, steps, leaf, e_ref, target, grid):
    """Largest tau in `grid` whose plain FP64 SP2 meets `target`; (tau, result)."""
    best = None
    for tau in sorted(grid):
        r = S.spamm_sp2(ctx, *csr, n_occ, steps, leaf, S.SPAMM_FP64, tau)
        if energy_error(r, e_ref) <= target:
            best = (tau, r)
        else:
            break
    return best


def calibrate_budget(ctx, mlp, csr, n_occ, steps, leaf, prec, e_ref, target, budgets, tau_min, tau_max,
                     margin: float = 10.0):
    """(largest budget in `budgets` whose learned-tau SP2 meets `target`) / margin, and
    the run at the largest passing budget; None if none passes."""
    best = None
    for b in sorted(budgets):
        r = S.spamm_sp2_learned(ctx, *csr, n_occ, steps, leaf, prec, mlp, b, tau_min, tau_max)
        if energy_error(r, e_ref) <= target:
            best = (b / margin, r)
        else:
            break
    return best


def calibrate_margin(ctx, mlp, csr, n_occ, steps, leaf, prec, e_ref, target, budgets, mu_refs, gains, tau_min,
                     tau_max, safety: float = 2.0):
    """The branch-margin rule's settings (budget, mu_ref, gain_max) with the fewest leaf
    products among those whose learned-tau SP2 (spamm_sp2_learned_margin) meets
    target / safety on a training system; (settings, run) or None."""
    best = None
    for b in budgets:
        for mu in mu_refs:
            for g in gains:
                r = S.spamm_sp2_learned_margin(ctx, *csr, n_occ, steps, leaf, prec, mlp, b, tau_min, tau_max, mu, g)
                if energy_error(r, e_ref) <= target / safety:
                    lp = int(sum(r["leaf_products"]))
                    if best is None or lp < best[2]:
                        best = ((b, mu, g), r, lp)
    return None if best is None else best[:2]
