"""Host pieces of bench.py that need no GPU: the roofline's DRAM traffic comes from a committed
ncu summary only while the kernel's source is the one that was profiled, and the equal-accuracy
comparison divides the right way."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_the_step_kernels_profile_matches_its_source():
    # the benchmark's dominant kernel: its committed counters describe the current source
    h = bench.kernel_src_hash("k_step3d7_z2(")
    traffic = bench.kernel_traffic("step3d7z2_fp32_sphere.json", h)
    assert traffic is not None and 150e6 < traffic < 300e6
    d = json.load(open(os.path.join(ROOT, "profiles", "step3d7z2_fp32_sphere.json")))
    assert d["algorithmic_bytes_per_launch"] == 16 * 16974593  # 16 B per node of the 257^3 grid


def test_changed_source_drops_the_traffic():
    assert bench.kernel_traffic("step3d7z2_fp32_sphere.json", "0" * 64) is None
    assert bench.kernel_traffic("no_such_profile.json", bench.kernel_src_hash("k_step3d7_z2(")) is None


def test_kernel_hash_reads_the_kernels_own_file():
    # kernels of step_pair.cu and step_bulk.cu are hashed from their own files
    assert bench.kernel_src_hash("k_step3d7_pair(") != bench.kernel_src_hash("k_step3d7_z2(")
    assert bench.kernel_src_hash("k_step3d7_bulk(") != bench.kernel_src_hash("k_step3d7_z2(")


def test_target_comparison():
    comps = {"fp64_plain": {"solves_per_s": 0.0131}, "fp64_tuned": {"solves_per_s": 0.0375}}
    out = bench.target_comparison(comps, 0.251, 3.0e-7)
    assert out["target_rel_err"] == 1e-6
    assert abs(out["speedup_vs_fp64_plain"] - 0.251 / 0.0131) < 1e-12
    assert abs(out["speedup_vs_fp64_tuned"] - 0.251 / 0.0375) < 1e-12
    assert bench.target_comparison({}, 0.25, 3e-7) is None
