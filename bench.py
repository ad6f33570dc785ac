"""SpAMM benchmark: dense-equivalent GFLOP/s of one GB300 on the algebraic-decay
workload (n = 8192, a_ij = u_ij / (|i-j|^3 + 1), leaf 64), with leaf-GEMM TFLOP/s and
roofline fractions.

One step = the whole hot path on one input: build the quadtree of A (norms of every
tier plus the leaf copies the precision needs, from the FP64 A resident in HBM), cull
the product space tier by tier, and sum the surviving leaf products of C = A A into
C's tiles and norms. A is symmetric, so C is: the output blocks i <= j are culled and
multiplied and the blocks i > j written as their transposes (SPAMM_SYM_PRODUCT).
Headline: tau = 1e-8, split-TF32 leaves (hi = tf32(a), lo = tf32(a - hi); the three
products hi hi + hi lo + lo hi on the tensor cores with FP32 accumulation), the
single-precision class of arithmetic the paper's leaves used.
A sweep over tau in {1e-10, 1e-8, 1e-6, 1e-4} and the leaf precisions reports each
one's time and its relative Frobenius error against the FP64 SpAMM on the GPU, one
compact line each, printed before the JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-sweep]
                  [--config alg8192 | lattice32768 | batched256 | sp2-32768]

--impl reference times the CPU oracle (plain FP64 recursive SpAMM) on this host.
Multi-GPU: every rank runs an independent replica (the products do not exchange data).
The other --config values measure the remaining workloads once, one JSON line each:
lattice32768 (n = 32768 physical-distance decay, FP16/BF16 leaves, leaf 64/128, three
tau), batched256 (256 exponential-decay matrices of uneven n in one launch under a CUDA
graph), sp2-32768 (SP2 on 32^3 tight-binding sites: fixed conservative tau in FP64
against the learned controller with split-TF32 leaves, errors against the stored
spectral reference).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N, LEAF, TAU = 8192, 64, 1e-8
HEADLINE = "tf32x3"
# nominal dense tensor rates per GPU (PFLOP/s): a precision's peak is the measured BF16
# peak times the ratio of its nominal rate to BF16's
NOMINAL_PF = {"bf16": 2.25, "fp16": 2.25, "tf32": 1.1}
TAUS = (1e-10, 1e-8, 1e-6, 1e-4)
WORKLOAD = "algebraic-decay n=8192 leaf=64 (a_ij=u_ij/(|i-j|^3+1), u=U[.5,1]*sign, seed 0)"
METRIC = "SpAMM dense-equiv GFLOP/s & leaf-GEMM % of TC peak at fixed error vs FP64 SpAMM"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return dict(hbm=p["hbm_gbs"], bf16=p["bf16_tflops"], bf16_sus=p["bf16_tflops_sustained"],
                    source="measured")
    except Exception:
        return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, source="fallback")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, device="cpu") -> float:
    """The largest of every rank's value (a time: the job ends with its slowest replica);
    the value itself outside a multi-rank process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job(per_replica_rate: float, ws: int) -> float:
    """Weak scaling, replicas only: every rank runs the whole workload, so the job's
    throughput is the replicas' count times the rate of the slowest one."""
    return per_replica_rate * ws


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()   # the sampler is live before the timed region starts
            while not self.lines and time.time() - t0 < 3.0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            k = len(self.lines)   # and takes one more sample after a timed region shorter than its period
            t0 = time.time()
            while len(self.lines) <= k and time.time() - t0 < 1.0:
                time.sleep(0.01)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash(parts) -> str:
    """First 16 hex digits of the SHA-256 of a kernel's source: each part is a file
    path relative to the repository, optionally cut to [begin marker, end marker)."""
    h = hashlib.sha256()
    for part in parts:
        text = open(os.path.join(ROOT, part["path"]), "rb").read()
        if "begin" in part:
            text = text[text.index(part["begin"].encode()):]
        if "end" in part:
            text = text[:text.index(part["end"].encode())]
        h.update(text)
    return h.hexdigest()[:16]


def kernel_traffic(name: str):
    """DRAM bytes per launch of `name` from the committed ncu summary, if the kernel's
    source is unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[name]
        if kernel_source_hash(rec["sources"]) != rec["sha256_16"]:
            return None
    except Exception:
        return None
    return rec["dram_bytes_per_launch"] * rec.get("scale", 1.0)


# ------------------------------------------------------------------ GPU arm

def run_gpu(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1011_3534_gb300 import spamm as S
    from paper_1011_3534_gb300 import workloads as W

    stream = torch.cuda.current_stream()
    ctx = S.spamm_ctx_create(local, stream, timing=True)
    A_host = W.algebraic_decay(N, 2, 0)
    dA = torch.from_numpy(A_host).to(f"cuda:{local}")
    pk = peaks()

    SYMP = S.SPAMM_SYM_PRODUCT   # A is symmetric: blocks i <= j multiplied, C_ji = C_ij^T

    def flags_for(prec):
        return S.COPY_FLAG[prec] | S.SPAMM_SYMMETRIC | S.SPAMM_NO_RIGHT

    def step(prec, tA, tC, tau, ev=None, mflags=0):
        if ev is not None:
            ev[0].record(stream)
        S.spamm_tree_update(tA, dA)                  # quadtree build (K1 + norm pyramid)
        if ev is not None:
            ev[1].record(stream)
        tC = S.spamm_multiply(ctx, tA, tA, tau, prec, SYMP | mflags, tC)   # cull + leaf products (+ mirror)
        if ev is not None:
            ev[2].record(stream)
        return tC

    def timed(prec, tau, steps, warmup, phases=True, mflags=0):
        tA = S.spamm_tree_build(ctx, dA, N, LEAF, flags_for(prec))
        tC = None
        for _ in range(warmup):
            tC = step(prec, tA, tC, tau, mflags=mflags)
        torch.cuda.synchronize()
        if phases:
            S.spamm_tree_build_ms(tA)   # start the leaf-block kernel's event count here
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        l0 = S.spamm_kernel_launches(ctx)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for s in range(steps):
            tC = step(prec, tA, tC, tau, evs[s] if phases else None, mflags)
        S.spamm_sync(ctx)   # the last product's norm pyramid (on its own stream) is inside the region
        t1.record(stream)
        torch.cuda.synchronize()
        launches = S.spamm_kernel_launches(ctx) - l0
        ms_total = max_over_ranks(t0.elapsed_time(t1), dA.device)
        ms_build = ms_mult = ms_k1 = None
        if phases:
            ms_k1 = S.spamm_tree_build_ms(tA)   # mean over the timed steps' K1 launches
            ms_build = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
            ms_mult = float(np.mean([e[1].elapsed_time(e[2]) for e in evs]))
        st = S.spamm_stats(tC)
        S.spamm_tree_free(tA)
        return dict(ms=ms_total / steps, ms_build=ms_build, ms_mult=ms_mult, ms_k1=ms_k1, stats=st,
                    launches=launches, tree=tC)

    # ---- headline
    prec = S.PRECISIONS[HEADLINE]
    for _ in range(1):
        r0 = timed(prec, TAU, 2, 1)   # allocate and warm caches
        S.spamm_tree_free(r0["tree"])
    with ClockSampler(local) as clk:
        r = timed(prec, TAU, args.steps, args.warmup)
    st = r["stats"]
    ms = r["ms"]
    dense_gflops = 2.0 * N ** 3 / (ms * 1e-3) / 1e9
    value = whole_job(dense_gflops, ws)
    # phase times inside the timed region (events on the library's stream)
    ms_leaf = st["ms_leaf"]
    ms_cull = st["ms_cull"]
    bytes_build = (8.0 + copy_bytes(HEADLINE)) * N * N   # read FP64 A, write the leaf copies
    build_gbs = bytes_build / (r["ms_k1"] * 1e-3) / 1e9   # K1 alone, from its own launch events
    # tensor work: the MMAs a triple needs in this precision (3 for the split forms)
    passes = 3 if HEADLINE.endswith("x3") else 1
    tc_flops = passes * st["leaf_flops"]
    tc_peak = pk["bf16_sus"] * NOMINAL_PF[HEADLINE[:4]] / NOMINAL_PF["bf16"]
    leaf_tflops = st["leaf_flops"] / (ms_leaf * 1e-3) / 1e12 if ms_leaf else None
    tc_tflops = tc_flops / (ms_leaf * 1e-3) / 1e12 if ms_leaf else None
    mma_tflops = st["mma_flops"] / (ms_leaf * 1e-3) / 1e12 if ms_leaf else None
    phases = {"build_ms": r["ms_build"], "k1_ms": r["ms_k1"], "cull_ms": ms_cull, "leaf_ms": ms_leaf,
              "multiply_ms": r["ms_mult"]}
    if r["ms_k1"] >= (ms_leaf or 0):
        roof = {"kernel": "k_tree_build", "bound": "hbm", "achieved": build_gbs, "peak": pk["hbm"],
                "unit": "GB/s", "frac": build_gbs / pk["hbm"],
                "traffic": kernel_traffic("k_tree_build"),
                "algorithmic_bytes_per_launch": bytes_build,
                "peak_source": pk["source"] + " hbm_gbs"}
    else:
        roof = {"kernel": "k_leaf_tc", "bound": "tensor", "achieved": tc_tflops,
                "peak": tc_peak, "unit": "TFLOP/s", "frac": tc_tflops / tc_peak,
                "traffic": kernel_traffic("k_leaf_tc"),
                "algorithmic_flops_per_launch": tc_flops,
                "peak_source": f"{pk['source']} bf16_tflops_sustained x {HEADLINE[:4]}/bf16 nominal"}
    # the leaf kernel's HBM floor: every leaf copy a computed triple reads, once, and
    # every block of C written (the mirrored ones included)
    lb = leaf_kernel_bytes(S.spamm_triples(r["tree"]), LEAF, copy_bytes(HEADLINE))
    leaf_gbs = lb["bytes"] / (ms_leaf * 1e-3) / 1e9 if ms_leaf else None
    leaf = {"useful_tflops": leaf_tflops, "tc_tflops": tc_tflops, "mma_issued_tflops": mma_tflops,
            "tc_peak": tc_peak, "frac_of_tc_peak": (tc_tflops / tc_peak) if tc_tflops else None,
            "leaf_products": st["leaf_products"], "mirrored_products": st["mirrored_products"],
            "hbm": {"algorithmic_bytes": lb["bytes"], "operand_leaves": lb["leaves"], "c_blocks": lb["blocks"],
                    "gbs": leaf_gbs, "frac": leaf_gbs / pk["hbm"] if leaf_gbs else None}}
    k1 = {"gbs": build_gbs, "frac_of_hbm": build_gbs / pk["hbm"], "bytes_per_launch": bytes_build}
    S.spamm_tree_free(r["tree"])

    # ---- end to end through the C ABI with host buffers (pinned): FP64 A in, FP32 C out
    A_pin = torch.from_numpy(A_host).pin_memory()
    C_pin = torch.empty((N, N), dtype=torch.float32).pin_memory()
    A_np, C_np = A_pin.numpy(), C_pin.numpy()
    tA = S.spamm_tree_build(ctx, A_np, N, LEAF, flags_for(prec))
    tC = None
    for _ in range(max(1, args.warmup)):
        S.spamm_tree_update(tA, A_np)
        tC = S.spamm_multiply(ctx, tA, tA, TAU, prec, SYMP, tC)
        S.spamm_tree_to_dense_f32(tC, C_np, asynchronous=True)
    S.spamm_sync(ctx)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 10))
    for _ in range(e2e_steps):
        # A goes in on the context's input copy stream and C comes back on its output
        # copy stream, so one step's output overlaps the next step's input
        S.spamm_tree_update(tA, A_np)
        tC = S.spamm_multiply(ctx, tA, tA, TAU, prec, SYMP, tC)
        S.spamm_tree_to_dense_f32(tC, C_np, asynchronous=True)
    S.spamm_sync(ctx)                        # every step's C is on the host
    e2e_ms = (time.perf_counter() - e0) * 1e3 / e2e_steps
    S.spamm_tree_free(tA)
    e2e_ms = max_over_ranks(e2e_ms, dA.device)
    S.spamm_tree_free(tC)
    e2e = {"value": whole_job(2.0 * N ** 3 / (e2e_ms * 1e-3) / 1e9, ws), "unit": "GFLOP/s",
           "h2d_bytes_per_step": 8 * N * N, "d2h_bytes_per_step": 4 * N * N, "ms_per_step": e2e_ms}

    # ---- precision and tau sweep (error vs FP64 SpAMM on the GPU)
    sweep = []
    if not args.no_sweep:
        for tau in TAUS:
            ref = None
            # "w": leaf 64 in warp tiles (SPAMM_WARP_TILES) instead of the tcgen05 items
            for name in ("fp64", "tf32", "bf16", "bf16x3", "tf32x3", "fp16", "bf16w", "tf32x3w"):
                p = S.PRECISIONS[name.rstrip("w")]
                rr = timed(p, tau, 3, 1, mflags=S.SPAMM_WARP_TILES if name.endswith("w") else 0)
                Cd = torch.empty((N, N), dtype=torch.float64, device=dA.device)
                S.spamm_tree_to_dense(rr["tree"], Cd)
                if name == "fp64":
                    ref = Cd
                    err = 0.0
                else:
                    err = float(torch.linalg.norm(Cd - ref) / torch.linalg.norm(ref))
                s2 = rr["stats"]
                sweep.append({"tau": tau, "prec": name, "ms": rr["ms"], "k1_ms": rr["ms_k1"],
                              "build_ms": rr["ms_build"], "cull_ms": s2["ms_cull"], "leaf_ms": s2["ms_leaf"],
                              "leaf_products": s2["leaf_products"], "err": err})
                S.spamm_tree_free(rr["tree"])
                del Cd
            del ref

    # ---- the shape autotuner's choice for the headline product (not timed)
    tuned = None
    if not args.no_sweep:
        tl, tf, tms = S.spamm_tune_shape(ctx, dA, N, TAU, prec, S.SPAMM_SYMMETRIC)
        tuned = {"leaf": tl, "tile": "warp 64x64" if tf else "tcgen05 items", "ms": tms,
                 "note": "build + product A A (full, not symmetric) per candidate"}

    # ---- CPU oracle on this host (rank 0 only, bounded sample, in a process of its own)
    cpu = cpu_baseline_subprocess(quick=args.no_sweep) if rank == 0 else None

    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": HEADLINE, "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "leaf": LEAF, "tau": TAU, "precision": HEADLINE,
                   "accumulate": "fp32 per pass", "product": "symmetric (blocks i <= j multiplied, i > j mirrored)",
                   "l2": "inputs larger than L2 (A is 512 MiB FP64)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "e2e": e2e, "gpu_launches": r["launches"], "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
        "phases": phases, "k1": k1, "leaf_gemm": leaf, "tuned_shape": tuned,
    }
    if rank == 0:
        for row in sorted(sweep, key=lambda x: (x["tau"] == TAU, x["tau"])):   # tau = 1e-8 last
            print(sweep_line(row))
        print(json.dumps(line, default=_compact))
    S.spamm_ctx_destroy(ctx)
    if ws > 1:
        dist.destroy_process_group()


def leaf_kernel_bytes(trip, leaf: int, elem_bytes: float) -> dict:
    """Algorithmic HBM bytes of one leaf-kernel launch of a symmetric product from its
    triple list (both halves listed): the leaf copies the computed triples (i <= j) read,
    A_ik at (i, k) and B_kj at (j, k) (rows of the symmetric operand), each once, and
    the FP32 blocks of C written, (i, j) and its mirror."""
    t = np.asarray(trip, dtype=np.int64)
    up = t[t[:, 0] <= t[:, 1]]
    leaves = np.unique(np.concatenate([up[:, 0] * 65536 + up[:, 2], up[:, 1] * 65536 + up[:, 2]])).size
    blocks = np.unique(t[:, 0] * 65536 + t[:, 1]).size
    return {"leaves": int(leaves), "blocks": int(blocks),
            "bytes": float(leaves * leaf * leaf * elem_bytes + blocks * leaf * leaf * 4)}


def copy_bytes(prec: str) -> float:
    """Bytes per element of the leaf copies a symmetric operand needs in `prec`."""
    return {"fp64": 8.0, "tf32": 4.0, "bf16": 2.0, "fp16": 2.0, "bf16x3": 4.0, "tf32x3": 8.0}[prec]


def sweep_line(row: dict) -> str:
    """One compact line per (tau, precision) of the sweep."""
    f = lambda v, d=4: "-" if v is None else f"{v:.{d}g}"
    return (f"sweep tau={row['tau']:.0e} {row['prec']:<6} step={f(row['ms'])}ms k1={f(row['k1_ms'])} "
            f"build={f(row['build_ms'])} cull={f(row['cull_ms'])} leaf={f(row['leaf_ms'])}ms "
            f"products={row['leaf_products']} err={f(row['err'], 2)}")


def _compact(o):
    return str(o)


# ------------------------------------------------------------------ CPU oracle

_ARM_PARTS = {0xd0c: "Neoverse-N1", 0xd40: "Neoverse-V1", 0xd49: "Neoverse-N2", 0xd4f: "Neoverse-V2",
              0xd8e: "Neoverse-N3", 0xd84: "Neoverse-V3"}


def host_cpu(cpuinfo_text=None):
    """The host CPU model: the x86 'model name' line of /proc/cpuinfo, or the Arm
    implementer and part numbers (named for the Neoverse cores), else the machine type."""
    import platform
    if cpuinfo_text is None:
        try:
            with open("/proc/cpuinfo") as f:
                cpuinfo_text = f.read()
        except OSError:
            cpuinfo_text = ""
    fields = {}
    for line in cpuinfo_text.splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            fields.setdefault(k.strip().lower(), v.strip())
    if fields.get("model name"):
        return fields["model name"]
    if "cpu part" in fields:
        try:
            impl, part = int(fields.get("cpu implementer", "0"), 16), int(fields["cpu part"], 16)
        except ValueError:
            return platform.machine()
        name = _ARM_PARTS.get(part, "") if impl == 0x41 else ""
        return f"{platform.machine()} implementer 0x{impl:02x} part 0x{part:03x}" + (f" ({name})" if name else "")
    return platform.machine()


def cpu_baseline(quick=False, budget_s=20.0):
    """The CPU oracle (FP64 recursive SpAMM, OpenMP over output quadrants) on the host
    cores: quadtree build + product at tau = 1e-8 on the full n = 8192 matrix, repeated
    while inside the time budget."""
    from paper_1011_3534_gb300 import workloads as W
    import oracle
    A_host = W.algebraic_decay(N, 2, 0)
    cores = oracle.max_threads()
    t0 = time.perf_counter()
    TA = oracle.Tree(A_host, LEAF)
    oracle.spamm(TA, TA, TAU, threads=cores)
    dt = time.perf_counter() - t0
    reps = 1
    if not quick:
        while (reps + 1) * dt < budget_s and reps < 5:
            t1 = time.perf_counter()
            TB = oracle.Tree(A_host, LEAF)
            oracle.spamm(TB, TB, TAU, threads=cores)
            dt = min(dt, time.perf_counter() - t1)
            reps += 1
    return {"value": 2.0 * N ** 3 / dt / 1e9, "unit": "GFLOP/s", "cores": cores, "cpu": host_cpu(), "kind": "oracle",
            "sample": f"full n={N} product at tau={TAU} (tree build + Eq. 4 recursion, FP64), best of {reps}, "
                      f"in a process of its own (no CUDA context)",
            "seconds": dt}


def cpu_baseline_subprocess(quick=False):
    """cpu_baseline() in a fresh interpreter, so that the oracle's threads share the host
    with no CUDA context or torch thread pool of the GPU process."""
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-baseline-child"] + (["--no-sweep"] if quick else [])
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
        return json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    except Exception as e:   # the GPU numbers stand without it
        return {"value": None, "unit": "GFLOP/s", "kind": "oracle", "error": f"{type(e).__name__}: {e}"}


def run_reference(args):
    """The CPU oracle on this host's cores, on the headline workload and metric. A step
    is the full product (tree build + Eq. 4 recursion) while K + W of them fit the time
    budget (SPAMM_REF_BUDGET_S, default 150 s); beyond that each step is a bounded
    sample: a seeded random set of the product's output blocks, each evaluated by the
    oracle's per-block recursion on all cores, with the tree of A built once before the
    timed steps, and the value is the dense-equivalent rate of the blocks computed. The
    line records the full product's rate from the sizing step beside it either way.
    --ref-n shrinks the matrix (tests of the mode switch only)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from concurrent.futures import ThreadPoolExecutor
    from paper_1011_3534_gb300 import workloads as W
    import oracle
    budget = float(os.environ.get("SPAMM_REF_BUDGET_S", "150"))
    n = args.ref_n or N
    A = W.algebraic_decay(n, 2, 0)
    cores = oracle.max_threads()

    def full_step():
        TA = oracle.Tree(A, LEAF)
        oracle.spamm(TA, TA, TAU, threads=cores)

    t0 = time.perf_counter()
    full_step()                                   # the first warm-up step, timed to size the rest
    t_full = time.perf_counter() - t0
    full_gflops = 2.0 * n ** 3 / t_full / 1e9
    per_step = budget / (args.steps + args.warmup)
    times = []
    if t_full <= per_step:
        for _ in range(args.warmup - 1):
            full_step()
        for _ in range(args.steps):
            t0 = time.perf_counter()
            full_step()
            times.append(time.perf_counter() - t0)
        ms = 1e3 * float(np.mean(times))
        v = 2.0 * n ** 3 / (ms * 1e-3) / 1e9
        mode = "full"
        sample = f"full n={n} product at tau={TAU} per step"
    else:
        TA = oracle.Tree(A, LEAF)
        nblk = TA.NB * TA.NB
        m = int(min(nblk, max(cores, per_step * nblk / t_full)))
        order = np.random.default_rng(7).permutation(nblk)
        with ThreadPoolExecutor(cores) as pool:
            def sample_step(s):
                idx = order[(s * m + np.arange(m)) % nblk]
                list(pool.map(lambda q: oracle.spamm_block(TA, TA, TAU, int(q) // TA.NB, int(q) % TA.NB), idx))

            for w in range(args.warmup - 1):
                sample_step(w)
            for s in range(args.steps):
                t0 = time.perf_counter()
                sample_step(args.warmup + s)
                times.append(time.perf_counter() - t0)
        ms = 1e3 * float(np.mean(times))
        v = 2.0 * n ** 3 * m / nblk / (ms * 1e-3) / 1e9
        mode = "sampled"
        sample = (f"{m} of {nblk} output blocks per step (seeded random order; Eq. 4 recursion per "
                  f"block on {cores} threads; tree of A built once before the timed steps), n={n}, "
                  f"tau={TAU}; a full step took {t_full:.2f} s")
    line = {"metric": METRIC, "value": v, "unit": "GFLOP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD if n == N else WORKLOAD.replace(f"n={N}", f"n={n}"), "n": n,
                       "leaf": LEAF, "tau": TAU, "precision": "fp64"},
            "cpu_baseline": {"value": v, "unit": "GFLOP/s", "cores": cores, "cpu": host_cpu(), "kind": "oracle",
                             "sample": sample, "mode": mode, "full_product_gflops": full_gflops},
            "e2e": {"value": v, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ other workloads

def _events_ms(stream, fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _line(config, value, ms, dtype, extra):
    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": 1, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic", "ms_per_step": ms,
            "config": config}
    line.update(extra)
    print(json.dumps(line))


def run_lattice(args):
    """n = 32768 physical-distance decay: each (leaf, precision, tau) timed as build +
    multiply from the resident FP64 matrix; errors against FP64 SpAMM on the GPU."""
    import torch
    from paper_1011_3534_gb300 import spamm as S
    from paper_1011_3534_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    ctx = S.spamm_ctx_create(0, stream, timing=True)
    A = torch.from_numpy(W.physical_decay(16, 8, 1.2, 0.1, 3, 1)).cuda()
    n = A.shape[0]
    rows = []
    with ClockSampler(0) as clk:
        for leaf in (64, 128):
            for tau in (1e-8, 1e-6, 1e-4):
                ref = None
                for name in ("fp64", "bf16", "fp16"):
                    if name == "fp64" and tau == 1e-8:
                        continue   # 4.6e13 FP64 flop: the error of this tau is not measured
                    p = S.PRECISIONS[name]
                    t = S.spamm_tree_build(ctx, A, n, leaf, S.COPY_FLAG[p] | S.SPAMM_SYMMETRIC | S.SPAMM_NO_RIGHT)
                    box = {}

                    def one():
                        S.spamm_tree_update(t, A)
                        box["c"] = S.spamm_multiply(ctx, t, t, tau, p, S.SPAMM_SYM_PRODUCT, box.get("c"))
                    ms = _events_ms(stream, one, 1 if name == "fp64" else min(args.steps, 5), 1 if name == "fp64" else 3)
                    st = S.spamm_stats(box["c"])
                    Cd = torch.empty((n, n), dtype=torch.float64, device=A.device)
                    S.spamm_tree_to_dense(box["c"], Cd)
                    if name == "fp64":
                        ref, err = Cd, 0.0
                    else:
                        err = float(torch.linalg.norm(Cd - ref) / torch.linalg.norm(ref)) if ref is not None else None
                        del Cd
                    rows.append({"leaf": leaf, "tau": tau, "prec": name, "ms_per_step": ms,
                                 "dense_equiv_gflops": 2.0 * n ** 3 / (ms * 1e-3) / 1e9,
                                 "leaf_ms": st["ms_leaf"], "cull_ms": st["ms_cull"],
                                 "leaf_tflops": st["leaf_flops"] / (st["ms_leaf"] * 1e-3) / 1e12 if st["ms_leaf"] else None,
                                 "mma_tflops": st["mma_flops"] / (st["ms_leaf"] * 1e-3) / 1e12 if st["ms_leaf"] else None,
                                 "leaf_products": st["leaf_products"], "rel_fro_err_vs_fp64_spamm": err})
                    S.spamm_tree_free(box["c"])
                    S.spamm_tree_free(t)
                del ref
    head = max((r for r in rows if r["prec"] != "fp64"), key=lambda r: r["dense_equiv_gflops"])
    _line({"workload": "physical-distance decay n=32768 (16^3 jittered lattice, 8 per site, exp(-1.2 r) N(0,1), seed 1)",
           "n": n, "leaf": head["leaf"], "tau": head["tau"], "precision": head["prec"], "accumulate": "fp32",
           "l2": "inputs larger than L2 (A is 8 GiB FP64)"},
          head["dense_equiv_gflops"], head["ms_per_step"], head["prec"],
          {"sweep": rows, "clocks": clk.summary()})
    S.spamm_ctx_destroy(ctx)


def run_batched(args):
    """256 symmetric exponential-decay matrices, n log-uniform in [512, 8192], tau = 1e-7,
    BF16 leaves: one step rebuilds the 256 trees (spread over the side streams) and runs
    the batched product (culls on side streams, one tensor-core launch per leaf size)
    from a CUDA graph."""
    import torch
    from paper_1011_3534_gb300 import spamm as S
    from paper_1011_3534_gb300 import workloads as W
    shapes = W.batched_shapes()
    tau, prec = 1e-7, S.SPAMM_BF16
    mats = [torch.from_numpy(W.batched_matrix(m, nm, lam)).cuda() for m, (nm, lam) in enumerate(shapes)]
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()   # graph capture needs a stream of its own
    ctx = S.spamm_ctx_create(0, stream)
    mid = sorted(range(len(shapes)), key=lambda m: shapes[m][0])[len(shapes) // 2]
    leaf, _ = S.spamm_tune_leaf(ctx, mats[mid], shapes[mid][0], tau, prec)
    fl = S.COPY_FLAG[prec] | S.SPAMM_SYMMETRIC | S.SPAMM_NO_RIGHT
    trees = [S.spamm_tree_build(ctx, X, X.shape[0], leaf, fl) for X in mats]
    dense = sum(2.0 * nm ** 3 for nm, _ in shapes)
    taus = np.full(len(trees), tau)
    box = {}

    def product_graph():
        box["C"] = S.spamm_multiply_batched(ctx, trees, trees, taus, prec, S.SPAMM_GRAPH, box.get("C"))

    def step():
        S.spamm_tree_update_batched(ctx, trees, mats)   # the 256 rebuilds side by side
        product_graph()

    def singles():
        box["C1"] = [S.spamm_multiply(ctx, t, t, tau, prec, 0, c) for t, c in zip(trees, box.get("C1") or [None] * len(trees))]

    with ClockSampler(0) as clk:
        k = min(args.steps, 20)
        ms_step = _events_ms(stream, step, k, args.warmup)
        ms_graph = _events_ms(stream, product_graph, k, args.warmup)
        ms_single = _events_ms(stream, singles, k, args.warmup)
    lp = sum(S.spamm_stats(c)["leaf_products"] for c in box["C"])
    _line({"workload": "256 exponential-decay matrices, n log-uniform [512, 8192], lambda U[0.7, 0.95], seed 3",
           "matrices": len(shapes), "sum_n2": int(sum(nm * nm for nm, _ in shapes)), "leaf": leaf, "tau": tau,
           "precision": "bf16", "accumulate": "fp32", "graph": True, "l2": "inputs larger than L2"},
          dense / (ms_step * 1e-3) / 1e9, ms_step, "bf16",
          {"batched_product_ms": ms_graph, "batched_product_dense_equiv_gflops": dense / (ms_graph * 1e-3) / 1e9,
           "one_launch_per_product_ms": ms_single, "leaf_products": lp,
           "leaf_tflops_over_product": lp * 2.0 * leaf ** 3 / (ms_graph * 1e-3) / 1e12, "clocks": clk.summary()})
    for c in box["C"] + box["C1"]:
        S.spamm_tree_free(c)
    for t in trees:
        S.spamm_tree_free(t)
    S.spamm_ctx_destroy(ctx)


def sp2_reference(side: int, seed: int = 2) -> dict:
    """The spectral SP2 reference of a tight-binding system, written by the CPU oracle
    (tests/golden/make_sp2_reference.py: dense FP64 eigensolve of H, then the TC2 steps
    applied to the spectrum)."""
    path = os.path.join(ROOT, "tests", "golden", "sp2_tb_spectral.json")
    return next(s for s in json.load(open(path))["systems"] if s["side"] == side and s["seed"] == seed)


def run_sp2(args):
    """SP2 on 32^3 tight-binding sites (n = 32768, 30 steps, leaf 64). Reference energy:
    the spectral SP2 of the dense FP64 eigensolve of H, stored by the CPU oracle. The
    fixed conservative tau is the largest of a half-decade grid whose split-TF32 SP2
    meets the 1e-6 target against that reference; plain FP64 SpAMM runs at it (the
    method without the controller, and its arbiter). The controller is trained and its
    budget calibrated on a 16^3 system (seed 7) and applied here without further
    calibration."""
    import torch
    from paper_1011_3534_gb300 import spamm as S
    from paper_1011_3534_gb300 import controller as CT
    from paper_1011_3534_gb300 import workloads as W
    ctx = S.spamm_ctx_create(0, torch.cuda.current_stream())
    steps, leaf, target = 30, 64, 1e-6
    small = W.tight_binding(16, seed=7)[:3]
    ns = 16 ** 3
    X, y = CT.collect(ctx, *small, ns / 2, steps, leaf, CT.half_decades(1e-12, 1e-3))
    m, loss = CT.train(ctx, X, y, epochs=1000)
    e_small = S.spamm_sp2(ctx, *small, ns / 2, steps, leaf, S.SPAMM_FP64, 0.0)["energy"]
    cal = CT.calibrate_budget(ctx, m, small, ns / 2, steps, leaf, S.SPAMM_TF32X3, e_small, target,
                              CT.half_decades(1e-8, 1e-3), 1e-12, 1e-3)
    budget = cal[0]
    calm = CT.calibrate_margin(ctx, m, small, ns / 2, steps, leaf, S.SPAMM_TF32X3, e_small, target,
                               CT.half_decades(1e-8, 1e-4), (3e-3, 1e-2, 3e-2, 1e-1), (10.0, 100.0), 1e-12, 1e-3)
    big = W.tight_binding(32, seed=2)[:3]
    n = 32 ** 3
    spec = sp2_reference(32)
    e_ref = spec["energy"]
    with ClockSampler(0) as clk:
        ref = S.spamm_sp2(ctx, *big, n / 2, steps, leaf, S.SPAMM_TF32X3, 1e-8)
        grid = {}
        for tau in CT.half_decades(1e-6, 1e-3):
            grid[tau] = S.spamm_sp2(ctx, *big, n / 2, steps, leaf, S.SPAMM_TF32X3, tau)
        ok = [t for t, r in grid.items() if CT.energy_error(r, e_ref) <= target]
        tau_c = max(t for t in ok if all(CT.energy_error(grid[u], e_ref) <= target for u in grid if u <= t)) if ok else 1e-6
        fixed_tc = grid[tau_c]
        fixed64 = S.spamm_sp2(ctx, *big, n / 2, steps, leaf, S.SPAMM_FP64, tau_c)
        learned = S.spamm_sp2_learned(ctx, *big, n / 2, steps, leaf, S.SPAMM_TF32X3, m, budget, 1e-12, 1e-3)
        margin = (S.spamm_sp2_learned_margin(ctx, *big, n / 2, steps, leaf, S.SPAMM_TF32X3, m, calm[0][0], 1e-12,
                                             1e-3, calm[0][1], calm[0][2]) if calm else None)
    dense = steps * 2.0 * n ** 3
    err = lambda r: CT.energy_error(r, e_ref)
    lp = lambda r: int(sum(r["leaf_products"]))
    head = margin if margin is not None else learned   # the learned form with the branch-margin budget
    _line({"workload": "SP2, 3-D tight binding on 32^3 sites (open boundaries, on-site U[-2,2], seed 2), "
                       "half filling, 30 steps", "n": n, "leaf": leaf,
           "precision": "tf32x3 (learned tau, branch-margin budget)" if margin is not None else "tf32x3 (learned tau)",
           "accumulate": "fp32 per pass", "tau_fixed": tau_c, "error_budget": budget,
           "reference": "spectral SP2 of the dense FP64 eigensolve of H (CPU oracle, stored)"},
          dense / (head["ms"] * 1e-3) / 1e9, head["ms"], "tf32x3",
          {"time_to_solution_ms": {"fp64_fixed_tau": fixed64["ms"], "tf32x3_fixed_tau": fixed_tc["ms"],
                                   "tf32x3_learned_tau": learned["ms"], "tf32x3_tau1e-8": ref["ms"]},
           "energy_rel_err_vs_reference": {"fp64_fixed_tau": err(fixed64), "tf32x3_fixed_tau": err(fixed_tc),
                                           "tf32x3_learned_tau": err(learned),
                                           "tf32x3_grid": {f"{t:.2e}": err(r) for t, r in grid.items()}},
           "arbiter_rel_diff_learned_vs_fp64_fixed_tau": abs(learned["energy"] - fixed64["energy"]) / abs(fixed64["energy"]),
           "tf32x3_tau1e-8_err_vs_reference": err(ref),
           "branches_equal_to_reference": {"fp64_fixed_tau": fixed64["branches"] == spec["branches"],
                                           "tf32x3_fixed_tau": fixed_tc["branches"] == spec["branches"],
                                           "tf32x3_learned_tau": learned["branches"] == spec["branches"]},
           "leaf_products": {"fp64_fixed_tau": lp(fixed64), "tf32x3_fixed_tau": lp(fixed_tc),
                             "tf32x3_learned_tau": lp(learned), "tf32x3_tau1e-8": lp(ref)},
           "learned_taus": learned["taus"], "controller_train_loss": loss, "clocks": clk.summary(),
           "margin_rule": None if margin is None else {
               "settings": {"budget": calm[0][0], "mu_ref": calm[0][1], "gain_max": calm[0][2]},
               "time_to_solution_ms": margin["ms"], "energy_rel_err_vs_reference": err(margin),
               "arbiter_rel_diff_vs_fp64_fixed_tau": abs(margin["energy"] - fixed64["energy"]) / abs(fixed64["energy"]),
               "leaf_products": lp(margin), "branches_equal_to_reference": margin["branches"] == spec["branches"]}})
    m.free()
    S.spamm_ctx_destroy(ctx)


def run_variants(args):
    """The threshold and dropping variants against plain SpAMM. (1) The depth-scaled
    threshold tau^{k+1} = tau^k / 8 (Sec. II) on the n = 8192 algebraic-decay product
    (BF16, leaf 64, symmetric product): step time, leaf products and error against the
    exact product. (2) SP2 on a 16^3 tight-binding system (n = 4096, 30 steps, leaf 64,
    FP64 products): SpAMM at tau against scheme (I), exact products filtered at tau
    (Sec. III), as energy error against dense SP2 (FP64 SpAMM at tau = 0) against the
    mean block products per step."""
    import torch
    from paper_1011_3534_gb300 import spamm as S
    from paper_1011_3534_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    ctx = S.spamm_ctx_create(0, stream, timing=True)
    N = 8192
    A = torch.from_numpy(W.algebraic_decay(N, 2, 0)).cuda()
    depth = []
    with ClockSampler(0) as clk:
        fl = S.COPY_FLAG[S.SPAMM_BF16] | S.SPAMM_SYMMETRIC | S.SPAMM_NO_RIGHT
        t = S.spamm_tree_build(ctx, A, N, 64, fl)
        t64 = S.spamm_tree_build(ctx, A, N, 64, S.SPAMM_KEEP_FP64 | S.SPAMM_SYMMETRIC)
        c0 = S.spamm_multiply(ctx, t64, t64, 0.0, S.SPAMM_FP64, S.SPAMM_SYM_PRODUCT)
        exact = torch.empty((N, N), dtype=torch.float64, device=A.device)
        S.spamm_tree_to_dense(c0, exact)
        S.spamm_tree_free(c0)
        S.spamm_tree_free(t64)
        for tau in (1e-8, 1e-6, 1e-4):
            for flags, name in ((0, "plain"), (S.SPAMM_DEPTH_TAU, "depth-scaled")):
                box = {}

                def one():
                    S.spamm_tree_update(t, A)
                    box["c"] = S.spamm_multiply(ctx, t, t, tau, S.SPAMM_BF16, S.SPAMM_SYM_PRODUCT | flags, box.get("c"))
                ms = _events_ms(stream, one, min(args.steps, 20), 3)
                st = S.spamm_stats(box["c"])
                Cd = torch.empty_like(exact)
                S.spamm_tree_to_dense(box["c"], Cd)
                err = float(torch.linalg.norm(Cd - exact) / torch.linalg.norm(exact))
                depth.append({"tau": tau, "threshold": name, "ms_per_step": ms,
                              "dense_equiv_gflops": 2.0 * N ** 3 / (ms * 1e-3) / 1e9,
                              "leaf_products": st["leaf_products"] + st["mirrored_products"],
                              "rel_fro_err_vs_exact": err})
                del Cd
                S.spamm_tree_free(box["c"])
        S.spamm_tree_free(t)
        del exact
        # SP2: SpAMM against scheme (I)
        ip, ix, d = W.tight_binding(16, seed=2)[:3]
        n = 16 ** 3
        ref = S.spamm_sp2(ctx, ip, ix, d, n / 2, 30, 64, S.SPAMM_FP64, 0.0)
        e_ref = ref["energy"]
        sp2 = []
        for tau in (1e-2, 3.16e-3, 1e-3, 3.16e-4, 1e-4, 3.16e-5, 1e-5, 1e-6):
            a = S.spamm_sp2(ctx, ip, ix, d, n / 2, 30, 64, S.SPAMM_FP64, tau)
            b = S.spamm_sp2_dropping(ctx, ip, ix, d, n / 2, 30, 64, S.SPAMM_FP64, tau)
            for name, r in (("spamm", a), ("dropping", b)):
                sp2.append({"tau": tau, "scheme": name, "energy_rel_err": abs(r["energy"] - e_ref) / abs(e_ref),
                            "mean_block_products": float(np.mean(r["leaf_products"])), "ms": r["ms"],
                            "branches_equal": r["branches"] == ref["branches"]})
        # site orderings: Morton (the default) against the Hilbert curve, same systems
        orders = []
        for order in ("morton", "hilbert"):
            ipo, ixo, do = W.tight_binding(16, seed=2, order=order)
            for tau in (1e-3, 1e-4, 1e-5):
                r = S.spamm_sp2(ctx, ipo, ixo, do, n / 2, 30, 64, S.SPAMM_FP64, tau)
                orders.append({"system": "sp2 16^3 fp64", "order": order, "tau": tau,
                               "energy_rel_err": abs(r["energy"] - e_ref) / abs(e_ref),
                               "mean_block_products": float(np.mean(r["leaf_products"])), "ms": r["ms"]})
        L = torch.from_numpy(W.physical_decay(16, 8, 1.2, 0.1, 3, 1)).cuda()
        perm = torch.from_numpy(W.site_permutation(16, "hilbert")).cuda()
        pb = (perm[:, None] * 8 + torch.arange(8, device=L.device)[None, :]).reshape(-1)
        nl = L.shape[0]
        for order in ("morton", "hilbert"):
            M = L if order == "morton" else L.index_select(0, pb).index_select(1, pb)
            t = S.spamm_tree_build(ctx, M, nl, 64, S.COPY_FLAG[S.SPAMM_BF16] | S.SPAMM_SYMMETRIC | S.SPAMM_NO_RIGHT)
            for tau in (1e-6, 1e-4):
                box = {}

                def one():
                    S.spamm_tree_update(t, M)
                    box["c"] = S.spamm_multiply(ctx, t, t, tau, S.SPAMM_BF16, S.SPAMM_SYM_PRODUCT, box.get("c"))
                ms = _events_ms(stream, one, 2, 1)
                st = S.spamm_stats(box["c"])
                orders.append({"system": "lattice n=32768 bf16", "order": order, "tau": tau, "ms_per_step": ms,
                               "leaf_products": st["leaf_products"] + st["mirrored_products"]})
                S.spamm_tree_free(box["c"])
            S.spamm_tree_free(t)
            del M
        del L
    head = max(depth, key=lambda r: r["dense_equiv_gflops"] if r["threshold"] == "depth-scaled" else 0)
    _line({"workload": "threshold and dropping variants: algebraic-decay n=8192 leaf=64 BF16 symmetric product; "
                       "SP2 16^3 tight-binding n=4096 leaf=64 FP64 (SpAMM vs scheme (I))",
           "n": N, "leaf": 64, "precision": "bf16", "accumulate": "fp32", "l2": "inputs larger than L2"},
          head["dense_equiv_gflops"], head["ms_per_step"], "bf16",
          {"depth_scaled": depth, "sp2_schemes": sp2, "orderings": orders, "sp2_reference_energy": e_ref,
           "sp2_reference_mean_block_products": float(np.mean(ref["leaf_products"])), "clocks": clk.summary()})
    S.spamm_ctx_destroy(ctx)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--ref-n", type=int, default=None, help=argparse.SUPPRESS)   # tests of the reference arm
    ap.add_argument("--cpu-baseline-child", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--config", default="alg8192",
                    choices=["alg8192", "lattice32768", "batched256", "sp2-32768", "variants"])
    args = ap.parse_args()
    if args.steps is None:   # the headline: a timed region of about 0.6 s; the oracle: 20 products
        args.steps = 20 if (args.impl == "reference" or args.config != "alg8192") else 2000
    if args.warmup < 3:
        args.warmup = 3
    if args.cpu_baseline_child:
        print(json.dumps(cpu_baseline(quick=args.no_sweep)))
    elif args.impl == "reference":
        run_reference(args)
    elif args.config == "lattice32768":
        run_lattice(args)
    elif args.config == "batched256":
        run_batched(args)
    elif args.config == "sp2-32768":
        run_sp2(args)
    elif args.config == "variants":
        run_variants(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
