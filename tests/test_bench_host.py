"""Host-side helpers of the benchmark that need no GPU: the CPU model recorded beside
the oracle's timing, read from /proc/cpuinfo on x86 and Arm hosts."""
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
