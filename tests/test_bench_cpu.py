"""CPU checks of bench.py: the work formulas, the digit-product count, the NUMA
helper without a GPU, and the reference arm's JSON line on the smallest workload."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_products_count_pairs_with_s_plus_t_below_S():
    for S in range(1, 9):
        pairs = sum(1 for s in range(S) for t in range(S) if s + t <= S - 1)
        assert bench.products(S) == pairs


def test_flops_follow_the_algorithmic_counts():
    w = dict(n_g=4000, n_v=128, n_c=2000, n_eig=400, n_freq=32)
    f = bench.flops(w)
    n_vc = 128 * 2000
    # Hermitian halves: chi0 4 N_G^2 N_vc, projection 8 N_eig N_G N_vc, chi_s 4 N_eig^2 N_vc N_w
    assert f["chi0"] == 4.0 * 4000 ** 2 * n_vc
    assert f["proj"] == 8.0 * 400 * 4000 * n_vc
    assert f["chis"] == 4.0 * 400 ** 2 * n_vc * 32
    assert abs(sum(f.values()) - 24.9e12) < 0.1e12


def test_gpu_local_cpus_without_a_gpu_is_none_or_allowed():
    cpus = bench.gpu_local_cpus(0)
    assert cpus is None or cpus <= os.sched_getaffinity(0)


def test_workloads_are_consistent():
    for name, w in bench.WORKLOADS.items():
        assert w["n_eig"] <= w["n_g"], name
        assert set(w) >= {"n_g", "n_v", "n_c", "n_eig", "n_freq"}, name


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "qpoint-400", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "q-points/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["config"]["workload"] == "qpoint-400"
