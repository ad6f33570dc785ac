"""Writes tests/golden/sp2_tb_spectral.json: the SP2 (TC2) reference of the cubic
tight-binding systems, from the CPU oracle only.

For each system (side^3 sites, open boundaries, nearest-neighbour hopping -1, on-site
energies U[-2, 2], Morton order, the seed given) the Hamiltonian's eigenvalues come
from the dense FP64 symmetric eigensolver (oracle.sp2.spectrum), and the trace-
correcting steps are applied to them (oracle.sp2.sp2_spectral: X commutes with H, so
every trace of the purification is a sum over the spectrum). Stored: the Gershgorin
interval, the energy Tr(H X_S) after 30 steps, the 31 traces and the 30 branches.
The paper prints no energies for these synthetic systems (its Figs. 4-6 use molecular
Fockians), so these are oracle values, not paper values.

Run: python tests/golden/make_sp2_reference.py [side ...]   (default: 16 32; the 32^3
system, n = 32768, needs about 17 GB of memory and a long dense eigensolve)
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import sp2 as O  # noqa: E402
from paper_1011_3534_gb300 import workloads as W  # noqa: E402

STEPS = 30
OUT = os.path.join(HERE, "sp2_tb_spectral.json")


def reference(side: int, seed: int) -> dict:
    ip, ix, d = W.tight_binding(side, seed=seed)[:3]
    n = side ** 3
    lo, hi = O.gershgorin(ip, ix, d, n)
    t0 = time.time()
    eigs = O.spectrum(ip, ix, d, n)
    secs = time.time() - t0
    r = O.sp2_spectral(eigs, n / 2, STEPS, lo, hi)
    return dict(side=side, seed=seed, n=n, n_occ=n / 2, steps=STEPS, emin=lo, emax=hi,
                energy=r["energy"], traces=r["traces"], branches=r["branches"],
                eig_min=float(eigs[0]), eig_max=float(eigs[-1]), eig_sum=float(eigs.sum()),
                eigensolve_seconds=round(secs, 1))


def main():
    sides = [int(a) for a in sys.argv[1:]] or [16, 32]
    try:
        rec = json.load(open(OUT))
    except (OSError, ValueError):
        rec = {"source": "spectral SP2 of the cubic tight-binding Hamiltonian (Sec. III TC2 purification); "
                         "eigenvalues by dense FP64 LAPACK, written by the CPU oracle", "systems": []}
    for side in sides:
        r = reference(side, 2)
        rec["systems"] = [s for s in rec["systems"] if not (s["side"] == side and s["seed"] == 2)] + [r]
        rec["systems"].sort(key=lambda s: (s["side"], s["seed"]))
        with open(OUT, "w") as f:
            json.dump(rec, f, indent=1)
            f.write("\n")
        print(f"side {side}: energy {r['energy']!r} ({r['eigensolve_seconds']} s)", flush=True)


if __name__ == "__main__":
    main()
