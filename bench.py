#!/usr/bin/env python
"""Benchmark of the static-subspace RPA hot path on GB300.

One step = every stage of one q-point through the C ABI: chi~(0), FP64
eigensolve and subspace basis, projection M~, chi_s(iw_k) for all k, the FP64
trace term, eigenvalues of every chi_s(iw_k) and E_c.  Workload: one q-point
with N_G=4000, N_v=128, N_c=2000 (N_vc=256000), N_eig=400, 32 frequencies,
synthetic splitmix64 matrix elements (16.4 GB complex128, larger than L2).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead (bounded sample, scaled to the workload).
Multi-GPU (torchrun): every rank runs its own q-point; no data-path collective.
"""
from __future__ import annotations

import argparse
import collections
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "q-points/sec and contraction TFLOP/s, mixed vs FP64 path at |dE_c|<=1e-6 Ha"
WORKLOADS = {
    "qpoint-4000": dict(n_g=4000, n_v=128, n_c=2000, n_eig=400, n_freq=32),
    "qpoint-400": dict(n_g=400, n_v=16, n_c=200, n_eig=40, n_freq=16),
    # small case for ncu captures (A is 0.5 GB, larger than L2)
    "qpoint-1024": dict(n_g=1024, n_v=32, n_c=1000, n_eig=128, n_freq=16),
    # the 4000-plane-wave q-point at the other subspace sizes of the mixed-precision study
    "qpoint-4000-neig200": dict(n_g=4000, n_v=128, n_c=2000, n_eig=200, n_freq=32),
    "qpoint-4000-neig800": dict(n_g=4000, n_v=128, n_c=2000, n_eig=800, n_freq=32),
    # the interface-sized q-point with complex64 matrix elements drawn on the device (50 GB)
    "qpoint-12000": dict(n_g=12000, n_v=256, n_c=2048, n_eig=1200, n_freq=48, m_dtype="c64"),
    # the same q-point with A never held whole: drawn again per chunk of 16 valence bands
    "qpoint-12000-streamed": dict(n_g=12000, n_v=256, n_c=2048, n_eig=1200, n_freq=48,
                                  m_dtype="c64", vc_chunk=16 * 2048),
}
# the uneven 4x4x4 q-grid: N_G in [1500, 6000], N_v = 96, N_c in [800, 2400], N_eig = N_G/10,
# 48 frequencies, every q-point's A drawn on the device; one step = all 64 q-points
BATCH_WORKLOADS = {"batch-64": dict(n_q=64, n_freq=48)}
# FP64 tensor/SIMT rate relative to dense BF16 (nominal 1.25 vs 2250 TFLOP/s)
FP64_OVER_BF16 = 1.25 / 2250.0
PRECISIONS = {"fp64": "RPA_FP64", "mixed": "RPA_MIXED", "bf16x3": "RPA_MIXED_BF16X3",
              "bf16x6": "RPA_MIXED_BF16X6", "tf32x3": "RPA_MIXED_TF32X3"}


def flops(w):
    n_vc = w["n_v"] * w["n_c"]
    return dict(chi0=4.0 * w["n_g"] ** 2 * n_vc,
                proj=8.0 * w["n_eig"] * w["n_g"] * n_vc,
                chis=4.0 * w["n_eig"] ** 2 * n_vc * w["n_freq"])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.bus = (bus_id or "").lower()
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out = self.proc.communicate(timeout=5)[0]
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = [r.split(", ") for r in getattr(self, "out", "").strip().splitlines() if r.count(",") >= 9]
        if not rows:
            return None
        tail = lambda b: b.strip().lower()[-7:]
        mine = [r for r in rows if self.bus and tail(r[1]) == tail(self.bus)]
        if not mine:
            mine = [r for r in rows if r[0] == rows[0][0]]
        sm = [float(r[2]) for r in mine if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in mine if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in mine for i in range(4) if r[6 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(mine)}


def setup_dist(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return rank, world, local, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(x, dist, device):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle leg (reported baseline; also the --impl reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(w, n_v_sample=4):
    """Time the FP64 oracle stage by stage on a sample of the workload: full N_G,
    N_eig and frequencies, n_v_sample of the N_v valence bands.  Stages linear in
    N_vc are scaled by N_v / n_v_sample; the two eigen-stages are not.
    Returns (seconds per full q-point, description, cores)."""
    import numpy as np
    import oracle.rpa_oracle as orc
    from paper_2405_20258_gb300 import inputs
    qp = inputs.make_qpoint(w["n_g"], n_v_sample, w["n_c"])
    A = inputs.matrix_elements(qp)
    delta = orc.transition_energies(qp.e_v, qp.e_c)
    t = {}
    t0 = time.perf_counter()
    chit = orc.chi_tilde(A, qp.qg2, delta, 0.0, qp.omega_cell)
    t["chi0"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    lam0, C, _ = orc.subspace_basis(chit, w["n_eig"])
    t["eig0"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    Mt = orc.project(A, qp.qg2, C)
    t["proj"] = time.perf_counter() - t0
    omega, weight = orc.frequency_grid(w["n_freq"])
    t["chis"] = t["eigs"] = 0.0
    for k in range(w["n_freq"]):
        t0 = time.perf_counter()
        cs = orc.chi_s(Mt, delta, omega[k], qp.omega_cell)
        orc.trace_term(Mt, delta, omega[k], qp.omega_cell)
        t1 = time.perf_counter()
        np.linalg.eigvalsh(0.5 * (cs + cs.conj().T))
        t["eigs"] += time.perf_counter() - t1
        t["chis"] += t1 - t0
    scale = w["n_v"] / n_v_sample
    est = (t["chi0"] + t["proj"] + t["chis"]) * scale + t["eig0"] + t["eigs"]
    measured = sum(t.values())
    desc = ("oracle stages on N_G=%d, N_v=%d of %d, N_c=%d, N_eig=%d, %d freq (%.1f s measured); "
            "vc-linear stages scaled x%g, eigensolves unscaled" %
            (w["n_g"], n_v_sample, w["n_v"], w["n_c"], w["n_eig"], w["n_freq"], measured, scale))
    return est, desc, os.cpu_count(), t


def reference_arm(args, w, rank, dist):
    if rank != 0:
        return
    steps = []
    t_all = None
    for s in range(args.warmup + args.steps):
        est, desc, cores, t = oracle_sample(w, n_v_sample=2)
        if s >= args.warmup:
            steps.append(est)
    sec = statistics.mean(steps)
    val = 1.0 / sec
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "q-points/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, **w},
            "cpu_baseline": {"value": val, "unit": "q-points/s", "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": val, "unit": "q-points/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

# DRAM traffic (read + write) of one chi~(0) slice_gemm launch at N_G = 4000 with K-blocks
# of 8,000 transitions and S = 4, from the ncu capture summarised in
# profiles/slice_gemm_chi0_ng4000.md (a K = 32,000 launch scaled to K = 16,000). Valid for
# the GEMM kernel as captured; set to None when the kernel changes until it is re-captured.
# The one change to slice_gemm since the capture moves a lone FP32 tail level into its own
# level's columns (S - Le == 1, the projection); the chi~(0) launch (S = 4, Le = 1) issues
# the same loads, MMAs and epilogue as captured.
CHI0_GEMM_TRAFFIC = {"workload": "qpoint-4000", "slices": 4, "bytes_per_launch": 3.52e9}


def products(S):
    """BF16 digit-product contractions per algorithmic one: pairs (s, t), s + t <= S - 1."""
    return S * (S + 1) // 2


def gpu_local_cpus(index):
    """CPUs on the GPU's NUMA node (from sysfs) that this process may run on, or None."""
    try:
        bus = subprocess.run(["nvidia-smi", "-i", str(index), "--query-gpu=pci.bus_id",
                              "--format=csv,noheader"], capture_output=True, text=True,
                             timeout=30).stdout.strip()
        dom, rest = bus.split(":", 1)
        path = "/sys/bus/pci/devices/%04x:%s/local_cpulist" % (int(dom, 16), rest.lower())
        cpus = set()
        for part in open(path).read().strip().split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        cpus &= os.sched_getaffinity(0)
        return cpus or None
    except Exception:
        return None


# Small cases for ncu captures of one kernel (a few GB on the device, inputs above L2):
#   chi0: the chi~(0) GEMM of a 4000-plane-wave q-point with 16,000 transitions (run with
#         RPA_TC_CHI0_BLOCKS=1 for one K-block of K = 32,000); chi0_static three times.
#   chis: the chi_s stage of a 1000-plane-wave q-point with 32,000 transitions, N_eig 400
#         and 4 frequencies; the whole chain twice.
#   eig:  the subspace stage (the library's eigensolver, FP32 start) of a 4000-plane-wave
#         q-point with 4,000 transitions (chi~ is the bench workload's size, A 0.26 GB);
#         chi0_static once, subspace_basis three times.
PROFILE_CASES = {
    "chi0": dict(n_g=4000, n_v=16, n_c=1000, n_eig=400, n_freq=8),
    "chis": dict(n_g=1000, n_v=16, n_c=2000, n_eig=400, n_freq=4),
    "eig": dict(n_g=4000, n_v=8, n_c=500, n_eig=400, n_freq=8),
}


def profile_case(name, slices):
    import torch
    from paper_2405_20258_gb300 import inputs, rpa
    w = PROFILE_CASES[name]
    qp = inputs.make_qpoint(w["n_g"], w["n_v"], w["n_c"])
    dq = rpa.device_qpoint(qp, w["n_eig"], w["n_freq"])
    A = torch.empty((w["n_v"] * w["n_c"], w["n_g"]), dtype=torch.complex128, device="cuda")
    rpa.rpa_generate_m(dq, 0, w["n_v"], 0, w["n_c"], A)
    torch.cuda.synchronize()
    dq.m = A
    sl = tuple(int(x) for x in slices.split(","))
    with rpa.Plan([dq], precision=rpa.RPA_MIXED, slices=sl, timing=True) as p:
        reps = 3 if name in ("chi0", "eig") else 2
        if name == "eig":
            p.chi0_static(0)
        for _ in range(reps):
            if name != "eig":
                p.chi0_static(0)
            if name in ("chis", "eig"):
                p.subspace_basis(0)
            if name == "chis":
                p.chi_freq(0)
        torch.cuda.synchronize()
        st, _ = p.timings()
    print(json.dumps({"profile": name, "case": w, "reps": reps,
                      "stage_ms": {k: v / reps for k, v in st.items() if v}}))


def run_steps(plan, n):
    return [plan.run(0) for _ in range(n)]


def batch_bench(args):
    """The uneven 64-q workload in one plan (rpa_ecorr over every q-point, inputs drawn
    on the device): q-points/s over `steps` passes, after `warmup` passes."""
    import torch
    from paper_2405_20258_gb300 import inputs, rpa
    w = BATCH_WORKLOADS["batch-64"]
    sizes = inputs.batched_workload()[:w["n_q"]]
    dqs = []
    for s in sizes:
        qp = inputs.make_qpoint(s["n_g"], s["n_v"], s["n_c"], iq=s["iq"],
                                q_twentieths=s["q_twentieths"])
        dqs.append(rpa.device_qpoint(qp, max(1, s["n_g"] // 10), w["n_freq"]))
    precision = getattr(rpa, PRECISIONS[args.precision])
    stream = torch.cuda.Stream()
    work = sum(sum(flops(dict(n_g=s["n_g"], n_v=s["n_v"], n_c=s["n_c"], n_eig=max(1, s["n_g"] // 10),
                              n_freq=w["n_freq"])).values()) for s in sizes)
    with rpa.Plan(dqs, precision=precision, stream=stream, timing=True) as p:
        for _ in range(args.warmup):
            p.ecorr(-1)
        p.timings()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler() as clk:
            e0.record(stream)
            for _ in range(args.steps):
                ecs = p.ecorr(-1)
            e1.record(stream)
            torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        st, launches = p.timings()
    line = {"metric": METRIC, "value": len(sizes) * args.steps / t, "unit": "q-points/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16" if args.precision != "fp64" else "f64",
            "data": "synthetic (splitmix64 matrix elements drawn on the device)",
            "config": {"workload": "batch-64", "n_q": len(sizes), "n_v": 96,
                       "n_g_range": [1500, 6000], "n_c_range": [800, 2400],
                       "n_eig": "N_G/10", "n_freq": w["n_freq"], "precision": args.precision,
                       "l2": "inputs larger than L2", "parallelism": "single GPU"},
            "contraction_tflops": work / (sum(st[k] for k in ("chi0", "proj", "chis")) / 1e3
                                          / args.steps) / 1e12,
            "stage_ms_per_step": {k: v / args.steps for k, v in st.items()},
            "gpu_launches": int(launches), "clocks": clk.summary(),
            "ec_ha_per_q": ecs}
    print(json.dumps(line), flush=True)


def plan_slices(precision, slices):
    """Digit planes per stage (chi~, projection, chi_s) the plan multiplies."""
    if precision in ("bf16x3", "tf32x3"):
        return (2, 2, 2)
    if precision == "bf16x6":
        return (3, 3, 3)
    return tuple(s if s > 0 else d for s, d in zip(slices, (4, 6, 3)))


def fp64_dgemm_tflops(dev):
    """Best of 5 float64 4096^3 matrix products (cuBLAS DGEMM through torch): the FP64
    peak the FP64 path's roofline is quoted against (a measurement, not a kernel of ours)."""
    try:
        import torch
        n = 4096
        a = torch.randn(n, n, dtype=torch.float64, device=dev)
        b = torch.randn(n, n, dtype=torch.float64, device=dev)
        torch.matmul(a, b)
        torch.cuda.synchronize(dev)
        best = None
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize(dev)
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
        del a, b
        return 2.0 * n ** 3 / best / 1e12
    except Exception:
        return None


def precision_study(w):
    """|dE_c| of each mixed precision against the FP64 path for the workload's q-point at
    N_eig 200, 400 and 800 (inputs drawn on the device; one JSON line per case)."""
    import torch
    from paper_2405_20258_gb300 import inputs, rpa
    qp = inputs.make_qpoint(w["n_g"], w["n_v"], w["n_c"])
    for n_eig in (200, 400, 800):
        if n_eig >= w["n_g"]:
            continue
        dq = rpa.device_qpoint(qp, n_eig, w["n_freq"])
        with rpa.Plan([dq], precision=rpa.RPA_FP64) as p:
            e64 = p.run(0)
        for name in ("mixed", "bf16x6", "bf16x3", "tf32x3"):
            with rpa.Plan([dq], precision=getattr(rpa, PRECISIONS[name]), timing=True) as p:
                ec = p.run(0)
                t0 = time.perf_counter()
                ec = p.run(0)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                st, _ = p.timings()
            print(json.dumps({"precision_study": name, "n_g": w["n_g"], "n_eig": n_eig,
                              "n_freq": w["n_freq"], "ec_fp64_ha": e64, "ec_ha": ec,
                              "abs_dEc_ha": abs(ec - e64), "rel_dEc": abs(ec - e64) / abs(e64),
                              "meets_1e-6_ha": abs(ec - e64) <= 1e-6, "ms_per_qpoint": dt * 1e3,
                              "contraction_ms": (st["chi0"] + st["proj"] + st["chis"]) / 2}),
                  flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="qpoint-4000",
                    choices=sorted(WORKLOADS) + sorted(BATCH_WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=sorted(PRECISIONS))
    ap.add_argument("--route", default="cholesky", choices=["eig", "cholesky"])
    ap.add_argument("--slices", default="4,6,3", help="digit slices of chi0, projection, chi_s")
    ap.add_argument("--no-chi0-diag", action="store_true",
                    help="mixed path: keep the sliced GEMM's diagonal of chi~ (no FP64 recompute)")
    ap.add_argument("--eig", default="own", choices=["own", "cusolver"],
                    help="eigensolver of chi~(0): the library's own (FP32 or FP64 tridiagonal "
                         "start, Cholesky-QR2, Rayleigh-Ritz by Jacobi), or cuSOLVER FP64")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile", default=None, choices=sorted(PROFILE_CASES),
                    help="run one stage of a small case three times (for ncu captures) and exit")
    ap.add_argument("--precision-study", action="store_true",
                    help="|dE_c| of every mixed precision against the FP64 path on the workload "
                         "at N_eig 200, 400 and 800 (one JSON line per case) and exit")
    args = ap.parse_args()
    if args.profile:
        profile_case(args.profile, args.slices)
        return
    if args.precision_study:
        precision_study(WORKLOADS[args.workload])
        return
    if args.workload in BATCH_WORKLOADS:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle's reference arm "
                              "times single q-point workloads"}))
            return
        batch_bench(args)
        return
    w = WORKLOADS[args.workload]
    if args.eig == "cusolver":
        os.environ["RPA_EIG"] = "cusolver"  # read by the library when a plan is created
    if args.no_chi0_diag:
        os.environ["RPA_TC_CHI0_DIAG"] = "0"  # read by the library at each chi~ stage
    rank, world, local, dist = setup_dist(args)
    if args.impl == "reference":
        reference_arm(args, w, rank, dist)
        if dist is not None:
            dist.destroy_process_group()
        return

    import numpy as np
    import torch
    from paper_2405_20258_gb300 import inputs, rpa

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rpa.load()
    mixed = args.precision != "fp64"
    precision = getattr(rpa, PRECISIONS[args.precision])
    if args.precision in ("bf16x3", "bf16x6", "tf32x3"):
        args.slices = "0,0,0"  # the split precisions fix their planes
    route = rpa.RPA_ROUTE_CHOLESKY if args.route == "cholesky" else rpa.RPA_ROUTE_EIG
    slices = tuple(int(x) for x in args.slices.split(","))
    stream = torch.cuda.Stream(device=dev)
    # each rank its own q-point of the 4x4x4 grid (weak scaling, no exchange)
    from paper_2405_20258_gb300.shard import qpoints_for_rank
    iq = qpoints_for_rank(64, rank % 64, min(world, 64))[0]
    qp = inputs.make_qpoint(w["n_g"], w["n_v"], w["n_c"], iq=iq,
                            q_twentieths=(1, 0, 0) if iq == 0 else inputs.qgrid_4x4x4()[iq])
    n_vc = w["n_v"] * w["n_c"]
    dq = rpa.device_qpoint(qp, w["n_eig"], w["n_freq"], device=dev)
    c64 = w.get("m_dtype") == "c64"
    A = torch.empty((n_vc, w["n_g"]), dtype=torch.complex64 if c64 else torch.complex128,
                    device=dev)
    if c64:
        dq.m_dtype = rpa.RPA_C64
    with torch.cuda.stream(stream):
        rpa.rpa_generate_m(dq, 0, w["n_v"], 0, w["n_c"], A, stream=stream)
    stream.synchronize()
    dq.m = A
    if w.get("vc_chunk"):
        args.no_e2e = True  # no host inputs to copy: A is drawn on the device per chunk
        dq.m = None  # drawn again per chunk by the library; A is never held whole
        del A
        A = torch.empty((0, w["n_g"]), dtype=torch.complex64, device=dev)
    plan = rpa.Plan([dq], precision=precision, energy_route=route, stream=stream, timing=True,
                    slices=slices if mixed else (0, 0, 0), vc_chunk=w.get("vc_chunk", 0))
    fl = flops(w)
    fl_total = sum(fl.values())

    ecs = run_steps(plan, args.warmup)
    plan.timings()
    torch.cuda.synchronize()
    barrier(dist)
    props = torch.cuda.get_device_properties(dev)
    bus = getattr(props, "pci_bus_id", None)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(bus) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        ecs += run_steps(plan, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    t_dev = ev0.elapsed_time(ev1) / 1e3
    stage_ms, launches = plan.timings()
    t_dev = max_over_ranks(t_dev, dist, dev)
    sec_per_step = t_dev / args.steps
    value = world * args.steps / t_dev
    contraction_s = (stage_ms["chi0"] + stage_ms["proj"] + stage_ms["chis"]) / 1e3 / args.steps
    contraction_tflops = fl_total / contraction_s / 1e12

    # roofline of the dominant contraction kernel
    pk, pk_kind = peaks()
    tot_ms = sum(stage_ms.values())
    shares = {k: v / tot_ms for k, v in stage_ms.items()}
    dom = max(("chi0", "proj", "chis"), key=lambda k: stage_ms[k])
    dom_s = stage_ms[dom] / 1e3 / args.steps
    fp64_peak = fp64_dgemm_tflops(dev)
    if mixed:
        eff = plan_slices(args.precision, slices)
        nprod = products(dict(chi0=eff[0], proj=eff[1], chis=eff[2])[dom])
        peak = pk["bf16_tflops_sustained"]
        achieved = fl[dom] * nprod / dom_s / 1e12
        traffic = None
        if (dom == "chi0" and CHI0_GEMM_TRAFFIC and args.workload == CHI0_GEMM_TRAFFIC["workload"]
                and slices[0] == CHI0_GEMM_TRAFFIC["slices"]):
            traffic = CHI0_GEMM_TRAFFIC["bytes_per_launch"]
        roofline = {"bound": "tensor", "kernel": "slice_gemm (%s)" % dom, "achieved": achieved,
                    "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "peak_source": "%s bf16 sustained (MEASURED_PEAKS.json)" % pk_kind,
                    "traffic": traffic,
                    "traffic_unit": "bytes per launch (ncu dram read + write)",
                    "work_per_step": "%d digit-product contractions x %.4g algorithmic flops, "
                    "all launches of the stage" % (nprod, fl[dom]),
                    # the method's own flops (one complex contraction) at the same time
                    "achieved_algorithmic": fl[dom] / dom_s / 1e12,
                    "frac_algorithmic": fl[dom] / dom_s / 1e12 / peak}
    else:
        peak = fp64_peak if fp64_peak else pk["bf16_tflops"] * FP64_OVER_BF16
        achieved = fl[dom] / dom_s / 1e12
        roofline = {"bound": "alu", "kernel": "fp64 %s" % dom, "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak,
                    "peak_source": ("measured: torch float64 matmul 4096^3 in this run (cuBLAS "
                                    "DGEMM), best of 5" if fp64_peak else
                                    "%s bf16 burst x nominal fp64/bf16 ratio (1.25/2250)" % pk_kind),
                    "traffic": None, "work_per_launch": "%.4g algorithmic flops" % fl[dom]}

    # end to end through the C ABI with host buffers: H2D of the step's inputs, E_c back.
    # Two input slots (two q-point entries of one plan over the same q-point): the copy of
    # step i+1's inputs into one slot runs on a copy stream while step i computes on the
    # other, as a stream of q-points would be fed.
    e2e = None
    if not args.no_e2e:
        plan.close()
        # pinned host buffers placed on the GPU's NUMA node: pages are placed where the
        # allocating thread runs, so the thread runs there while it allocates them
        saved = os.sched_getaffinity(0)
        near = gpu_local_cpus(local)
        if near:
            os.sched_setaffinity(0, near)
        host_A = torch.empty(A.shape, dtype=A.dtype, pin_memory=True)
        host_small = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
                      for t in (dq.qg2, dq.e_v, dq.e_c)]
        os.sched_setaffinity(0, saved)
        host_A.copy_(A)
        for h_, t in zip(host_small, (dq.qg2, dq.e_v, dq.e_c)):
            h_.copy_(t)
        h2d = host_A.numel() * host_A.element_size() + sum(t.numel() * t.element_size()
                                                          for t in host_small)
        dq2 = rpa.device_qpoint(qp, w["n_eig"], w["n_freq"], device=dev)
        dq2.m = torch.empty_like(A)
        slots = [dq, dq2]
        plan_e = rpa.Plan(slots, precision=precision, energy_route=route, stream=stream,
                          timing=True, slices=slices if mixed else (0, 0, 0))
        copy_stream = torch.cuda.Stream(device=dev)
        ready = [torch.cuda.Event(), torch.cuda.Event()]
        h2d_ev = []

        def stage(i, after=None):
            # H2D of step i's inputs into slot i % 2 (its previous user, step i-2, is done:
            # plan.run returns only after the step's result reached the host), all pieces
            # queued on the copy stream at once: the copy engine then runs at the link's
            # rate beside the running step, whose own small device-to-host reads wait at
            # most one piece's length (64 MB: 0.3 ms at 210 GB/s, 2 ms at 35 GB/s; host links
            # have been measured at both rates)
            d = slots[i % 2]
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            rows = max(1, (64 << 20) // (host_A.shape[1] * host_A.element_size()))
            with torch.cuda.device(dev), torch.cuda.stream(copy_stream):
                if after is not None:
                    copy_stream.wait_event(after)
                c0.record(copy_stream)
                for r0 in range(0, host_A.shape[0], rows):
                    d.m[r0:r0 + rows].copy_(host_A[r0:r0 + rows], non_blocking=True)
                for d_, h_ in zip((d.qg2, d.e_v, d.e_c), host_small):
                    d_.copy_(h_, non_blocking=True)
                c1.record(copy_stream)
                ready[i % 2].record(copy_stream)
            h2d_ev.append((c0, c1))

        host_ms = collections.defaultdict(float)

        def timed(name, fn, *a):
            t0 = time.perf_counter()
            r = fn(*a)
            host_ms[name] += (time.perf_counter() - t0) * 1e3
            return r

        def run_e2e(n, after=None):
            stage(0, after)
            ecs_e = []
            for i in range(n):
                stream.wait_event(ready[i % 2])
                # the stages of step i through the public API; step i+1's inputs are
                # queued as soon as chi~(0) of step i is queued, and copy during the whole
                # step: no stage after that puts a host-to-device copy on the copy engine
                # (the transition sort runs on the device, the eigensolver's cluster starts
                # reach it as kernel arguments), so none waits behind the 16 GB copy
                timed("chi0_static", plan_e.chi0_static, i % 2)
                if i + 1 < n:
                    timed("stage", stage, i + 1)
                timed("subspace_basis", plan_e.subspace_basis, i % 2)
                timed("chi_freq", plan_e.chi_freq, i % 2)
                ecs_e.append(timed("ecorr", plan_e.ecorr, i % 2))  # E_c to the host (8 bytes)
            return ecs_e

        run_e2e(2)
        torch.cuda.synchronize()
        plan_e.timings()
        h2d_ev.clear()
        host_ms.clear()
        barrier(dist)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ecs_e2e = run_e2e(args.steps, after=e0)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(dist)
        t_e2e = max_over_ranks(e0.elapsed_time(e1) / 1e3, dist, dev)
        e2e_stage_ms, _ = plan_e.timings()
        h2d_ms = [a.elapsed_time(b) for a, b in h2d_ev]
        e2e = {"value": world * args.steps / t_e2e, "unit": "q-points/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 8,
               "h2d_ms_per_step": statistics.mean(h2d_ms),
               "h2d_overlap": "step i+1's inputs are copied during step i (two input slots)",
               "host_buffers": "pinned, allocated by a thread on the GPU's NUMA node" if near
               else "pinned",
               "ec_spread": max(ecs_e2e) - min(ecs_e2e),
               "stage_ms_per_step": {k: v / args.steps for k, v in e2e_stage_ms.items()},
               "host_ms_per_call": {k: v / args.steps for k, v in host_ms.items()}}
        plan_e.close()
        del host_A, dq2, slots

    # the FP64 path on the same inputs: speed-up and |dE_c| of the mixed path
    compare = None
    if mixed and not args.no_fp64_compare:
        p64 = rpa.Plan([dq], precision=rpa.RPA_FP64, energy_route=route, stream=stream, timing=True)
        run_steps(p64, 1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ec64 = run_steps(p64, 1)[0]
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        st64, _ = p64.timings()
        p64.close()
        compare = {"fp64_q_per_s": 1.0 / t64, "fp64_ms_per_step": t64 * 1e3, "fp64_ec_ha": ec64,
                   "mixed_ec_ha": ecs[-1], "abs_dEc_ha": abs(ecs[-1] - ec64),
                   "rel_dEc": abs(ecs[-1] - ec64) / abs(ec64), "speedup": t64 / sec_per_step,
                   "contraction_speedup": ((st64["chi0"] + st64["proj"] + st64["chis"]) / 1e3)
                   / contraction_s,
                   "fp64_steps": 1, "fp64_warmup": 1}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        est, desc, cores, _ = oracle_sample(w)
        cpu = {"value": 1.0 / est, "unit": "q-points/s", "cores": cores, "kind": "oracle",
               "sample": desc}

    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": "q-points/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec_per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if mixed else "f64",
        "data": "synthetic (splitmix64 matrix elements drawn on the device)",
        "config": {"workload": args.workload, **w, "n_vc": n_vc, "precision": args.precision,
                   "slices": list(slices) if mixed else None, "energy_route": args.route,
                   "eigensolver": args.eig,
                   "chi0_fp64_diagonal": (not args.no_chi0_diag) if mixed else None,
                   "l2": ("inputs larger than L2 (A is %.1f GB, drawn per chunk of %d transitions, "
                          "never whole)" % (n_vc * w["n_g"] * (8 if c64 else 16) / 1e9, w["vc_chunk"])
                          if w.get("vc_chunk") else
                          "inputs larger than L2 (A is %.1f GB)" % (A.numel() * A.element_size() / 1e9)),
                   "parallelism": "one q-point per GPU" if world > 1 else "single GPU"},
        "contraction_tflops": contraction_tflops,
        "stage_ms_per_step": {k: v / args.steps for k, v in stage_ms.items()},
        "stage_share": shares,
        "roofline": roofline,
        "mixed_vs_fp64": compare,
        "fp64_peak_tflops_measured": fp64_peak,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "ec_ha": ecs[-1], "ec_spread_over_steps": max(ecs) - min(ecs),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
