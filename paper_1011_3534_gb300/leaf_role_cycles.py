"""Per-role cycle counts of the tensor-core leaf kernel (a profiling probe).

Builds the library with -DSPAMM_LEAF_ROLE_CYCLES into _build_roles/ (the library's own
build is not touched), runs one product of the benchmark's workload per precision
(n = 8192 algebraic decay, leaf 64, tau = 1e-8, symmetric operand and product) on that
build, and prints, per CTA on average, the cycles each role of `k_leaf_tc` spends:

  producer  (TMA, warp 0)     total, waiting for a free stage
  MMA       (warp 1)          total, waiting for a stage's data, waiting for a free
                              accumulator, issuing tcgen05.mma (per stage)
  epilogue  (warps 2-5)       total, waiting for a finished accumulator, storing C and
                              its norms
  item hand-off               MMA and epilogue waiting for the next item, producer
                              publishing it and reading the next item's description

and the spread of the CTAs' totals (load balance).

  python -m paper_1011_3534_gb300.leaf_role_cycles [n] [alg|lattice]

(lattice: the n = 32768 physical-distance-decay matrix at tau = 1e-6, whose near-dense
products give items of up to hundreds of passes.)
"""
from __future__ import annotations

import ctypes
import os
import sys

import numpy as np


def main(n: int = 8192, workload: str = "alg"):
    import torch
    from . import build as B
    B.build()                       # the library's own build, which the binding loads on import
    from . import spamm as S
    from . import workloads as W
    so = B.build(extra=["-DSPAMM_LEAF_ROLE_CYCLES"], out_dir=os.path.join(B.HERE, "_build_roles"))
    L = ctypes.CDLL(so)
    S._declare(L)
    S.LIB = L                       # the probe build in place of the library's own
    L.spamm_leaf_role_cycles.argtypes = [ctypes.c_void_p, ctypes.c_int]
    ctx = S.spamm_ctx_create(0, torch.cuda.current_stream(), timing=True)
    if workload == "lattice":   # n = 32768 physical-distance decay, near-dense products
        A = torch.from_numpy(W.physical_decay(16, 8, 1.2, 0.1, 3, 1)).cuda()
        n = A.shape[0]
    else:
        A = torch.from_numpy(W.algebraic_decay(n, 2, 0)).cuda()
    tau = 1e-6 if workload == "lattice" else 1e-8
    for name in ("tf32x3", "bf16", "bf16x3"):
        p = S.PRECISIONS[name]
        t = S.spamm_tree_build(ctx, A, n, 64, S.COPY_FLAG[p] | S.SPAMM_SYMMETRIC | S.SPAMM_NO_RIGHT)
        C = S.spamm_multiply(ctx, t, t, tau, p, S.SPAMM_SYM_PRODUCT)   # warm-up
        S.spamm_sync(ctx)
        L.spamm_leaf_role_cycles(None, 1)
        C = S.spamm_multiply(ctx, t, t, tau, p, S.SPAMM_SYM_PRODUCT, C)
        st = S.spamm_stats(C)
        buf = np.zeros((1024, 16), dtype=np.uint64)
        L.spamm_leaf_role_cycles(buf.ctypes.data, 0)
        grid = int(torch.cuda.get_device_properties(0).multi_processor_count)
        b = buf[:grid].astype(np.float64)
        stages = b[:, 9].sum()
        print(f"{name}: leaf {st['ms_leaf'] * 1e3:.1f} us, {b[:, 8].sum():.0f} items, {stages:.0f} stages; "
              f"per CTA (cycles): producer {b[:, 1].mean():.0f} (waiting for a stage {b[:, 0].mean():.0f}); "
              f"MMA {b[:, 5].mean():.0f} (waiting for data {b[:, 2].mean():.0f}, for an accumulator "
              f"{b[:, 3].mean():.0f}, issuing {b[:, 4].mean():.0f} = {b[:, 4].sum() / max(stages, 1):.0f} per stage); "
              f"epilogue {b[:, 7].mean():.0f} (waiting {b[:, 6].mean():.0f}); CTA totals max/mean "
              f"{b[:, 7].max() / max(b[:, 7].mean(), 1):.2f}", flush=True)
        print(f"  item hand-off (cycles per CTA): MMA waiting for the next item {b[:, 10].mean():.0f}, "
              f"epilogue waiting for the next item {b[:, 14].mean():.0f}; producer publishing "
              f"{b[:, 11].mean():.0f}, describing the next item {b[:, 12].mean():.0f}; epilogue stores and "
              f"norms {b[:, 13].mean():.0f}", flush=True)
        S.spamm_tree_free(C)
        S.spamm_tree_free(t)
    S.spamm_ctx_destroy(ctx)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 8192, sys.argv[2] if len(sys.argv) > 2 else "alg")
