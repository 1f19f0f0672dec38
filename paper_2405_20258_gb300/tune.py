"""Autotuner of the tensor-core GEMM pipeline for one problem shape.

The GEMM's pipeline shape is read from environment knobs when a plan runs:
RPA_TC_NA (A-ring slots), RPA_TC_NB (B buffers), RPA_TC_NACC (TMEM accumulator
sets), RPA_TC_GROUP (tile rows per rasterisation group), RPA_TC_GRID (persistent
grid), RPA_TC_CHIS_GROUP (frequencies per chi_s launch).  This tool times every
candidate setting on device-drawn inputs of the given shape, each in a fresh
process (so the knobs are read anew), and prints the fastest as a JSON line of
environment assignments:

    python -m paper_2405_20258_gb300.tune --shape 4000,128,2000,400,32 --slices 4,6,3

It runs the mixed path only; every candidate must reproduce the default E_c to
1e-10 relative (the knobs change the schedule, not the arithmetic).
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CANDIDATES = {
    "RPA_TC_NB": ["2", "3"],
    "RPA_TC_GROUP": ["4", "8", "16"],
}


def child(shape, slices, reps):
    import torch
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_2405_20258_gb300 import inputs, rpa
    n_g, n_v, n_c, n_eig, n_freq = shape
    qp = inputs.make_qpoint(n_g, n_v, n_c)
    dq = rpa.device_qpoint(qp, n_eig, n_freq)
    A = torch.empty((n_v * n_c, n_g), dtype=torch.complex128, device="cuda")
    rpa.rpa_generate_m(dq, 0, n_v, 0, n_c, A)
    torch.cuda.synchronize()
    dq.m = A
    with rpa.Plan([dq], precision=rpa.RPA_MIXED, slices=slices, timing=True) as p:
        ec = p.run(0)
        p.timings()
        for _ in range(reps):
            ec = p.run(0)
        st, _ = p.timings()
    gemm = sum(st[k] for k in ("chi0", "proj", "chis", "slice")) / reps
    print(json.dumps({"ec": ec, "gemm_ms": gemm,
                      "stages": {k: v / reps for k, v in st.items() if v}}))


def run_candidate(setting, a):
    """Time one knob setting in a fresh process; its JSON line, or {"error": ...}."""
    env = dict(os.environ)
    env.update(setting)
    r = subprocess.run([sys.executable, "-m", "paper_2405_20258_gb300.tune", "--child",
                        "--shape", a.shape, "--slices", a.slices, "--reps", str(a.reps)],
                       env=env, capture_output=True, text=True, cwd=os.path.dirname(HERE))
    if r.returncode != 0:
        return {"error": r.stderr.strip()[-300:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def select(grid, run):
    """Run the default setting and every point of the grid (knob -> values) through
    run(setting); the fastest candidate whose E_c equals the default's to 1e-10
    relative wins.  Returns (best or None, all results)."""
    keys = list(grid)
    results = []
    base_ec = None
    for values in [None] + list(itertools.product(*(grid[k] for k in keys))):
        setting = {} if values is None else dict(zip(keys, values))
        out = run(setting)
        if "error" in out:
            results.append({"env": setting, "error": out["error"]})
            continue
        if base_ec is None:
            base_ec = out["ec"]
        out = dict(out)
        out["agrees"] = abs(out["ec"] - base_ec) <= 1e-10 * abs(base_ec)
        results.append({"env": setting, **out})
    ok = [r for r in results if "gemm_ms" in r and r["agrees"]]
    return (min(ok, key=lambda r: r["gemm_ms"]) if ok else None), results


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--shape", default="4000,128,2000,400,32",
                    help="n_g,n_v,n_c,n_eig,n_freq")
    ap.add_argument("--slices", default="4,6,3")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--grid", default=None,
                    help='JSON object of knob -> list of values (default: %s)' % json.dumps(CANDIDATES))
    ap.add_argument("--child", action="store_true", help=argparse.SUPPRESS)
    a = ap.parse_args(argv)
    shape = tuple(int(x) for x in a.shape.split(","))
    slices = tuple(int(x) for x in a.slices.split(","))
    if a.child:
        child(shape, slices, a.reps)
        return
    grid = json.loads(a.grid) if a.grid else CANDIDATES

    def run(setting):
        out = run_candidate(setting, a)
        print(json.dumps({"env": setting, **out}), file=sys.stderr, flush=True)
        return out

    best, results = select(grid, run)
    print(json.dumps({"shape": shape, "slices": slices, "best_env": best and best["env"],
                      "best_gemm_ms": best and best["gemm_ms"],
                      "default_gemm_ms": results[0].get("gemm_ms"),
                      "candidates": len(results)}))


if __name__ == "__main__":
    main()
