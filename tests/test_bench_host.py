"""Host-side helpers of the benchmark that need no GPU: the CPU model recorded beside
the oracle's timing, the clock-sample summary, and the kernel-source hash that keeps a
recorded DRAM traffic figure only while the kernel is unchanged."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

X86 = "processor\t: 0\nvendor_id\t: GenuineIntel\nmodel name\t: Example CPU @ 2.70GHz\nflags\t\t: fpu\n"
ARM = ("processor\t: 0\nBogoMIPS\t: 2000.00\nFeatures\t: fp asimd\nCPU implementer\t: 0x41\n"
       "CPU architecture: 8\nCPU variant\t: 0x0\nCPU part\t: 0xd4f\nCPU revision\t: 0\n")


def test_x86_model_name():
    assert bench.host_cpu(X86) == "Example CPU @ 2.70GHz"


def test_arm_implementer_and_part():
    s = bench.host_cpu(ARM)
    assert "implementer 0x41" in s and "part 0xd4f" in s and s.endswith("(Neoverse-V2)")


def test_unknown_part_and_empty_text():
    s = bench.host_cpu(ARM.replace("0xd4f", "0x123"))
    assert "part 0x123" in s and "(" not in s
    assert bench.host_cpu("") and bench.host_cpu("garbage without fields")


def test_this_host():
    assert isinstance(bench.host_cpu(), str) and bench.host_cpu()


def test_clock_summary_parses_samples():
    c = bench.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
               "0, 1965, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 950.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
               "garbage", ""]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3


def test_clock_summary_without_samples():
    s = bench.ClockSampler(0).summary()
    assert s["sm_mhz"] is None and s["samples"] == 0


def test_kernel_hash_covers_only_the_marked_region(tmp_path):
    f = tmp_path / "k.cu"
    f.write_text("head\n// BEGIN\nbody\n// END\ntail\n")
    part = [{"path": str(f), "begin": "// BEGIN", "end": "// END"}]
    h0 = bench.kernel_source_hash(part)
    f.write_text("other head\n// BEGIN\nbody\n// END\nother tail\n")
    assert bench.kernel_source_hash(part) == h0
    f.write_text("head\n// BEGIN\nchanged body\n// END\ntail\n")
    assert bench.kernel_source_hash(part) != h0


def test_traffic_of_unknown_kernel_is_null():
    assert bench.kernel_traffic("no_such_kernel") is None


def _reference_line(n, steps, warmup, budget):
    import json
    import subprocess
    env = dict(os.environ, OMP_NUM_THREADS="4", SPAMM_REF_BUDGET_S=str(budget))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", str(steps),
                        "--warmup", str(warmup), "--ref-n", str(n)], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])


def test_reference_arm_samples_when_the_steps_exceed_its_budget():
    # n = 2048 (NB = 32): a full product takes well under a second, a 0.05 s budget
    # forces the sampled mode
    d = _reference_line(2048, 10, 3, 0.05)
    assert d["impl"] == "reference" and d["steps"] == 10 and d["value"] > 0
    assert d["cpu_baseline"]["mode"] == "sampled"
    assert "output blocks per step" in d["cpu_baseline"]["sample"]


def test_reference_arm_modes_agree():
    # the per-block sample and the full product measure the same dense-equivalent rate:
    # the sampled blocks run the same recursion, followed into one output block each.
    # A 1 s budget over 6 steps samples about a quarter of the 1024 blocks per step, so
    # the threads stay balanced; a factor of 1.5 either way allows for the full
    # product's tree build and a shared host (measured: within 10%)
    full = _reference_line(2048, 3, 3, 1e6)
    samp = _reference_line(2048, 3, 3, 1.0)
    assert full["cpu_baseline"]["mode"] == "full" and samp["cpu_baseline"]["mode"] == "sampled"
    ratio = samp["value"] / full["value"]
    assert 1 / 1.5 < ratio < 1.5, ratio


def test_leaf_kernel_bytes_counts_each_leaf_and_block_once():
    # triples of a symmetric product, both halves listed: (0,1,0) and its mirror (1,0,0),
    # the diagonal (1,1,0) and (1,1,1). Computed (i <= j): reads A_00, B at (1,0); A_10,
    # B at (1,0); A_11, B at (1,1) -> copies (0,0), (1,0), (1,1); blocks (0,1), (1,0), (1,1)
    import bench
    trip = [(0, 1, 0), (1, 0, 0), (1, 1, 0), (1, 1, 1)]
    r = bench.leaf_kernel_bytes(trip, 64, 8.0)
    assert r["leaves"] == 3 and r["blocks"] == 3
    assert r["bytes"] == 3 * 64 * 64 * 8 + 3 * 64 * 64 * 4
