"""Parity cases at the sizes of the other workload configurations.

* N_G = 400 with N_eig = 200: the default mixed path within 1e-6 Ha of the oracle.
* N_G = 4000, N_v = 128, N_c = 2000, 32 frequencies with N_eig in {200, 400, 800}:
  the default mixed path against the FP64 CUDA path on the same device-drawn inputs
  (the oracle cannot run this size in a test); the error is stated per N_eig.
* The uneven multi-q batch (4x4x4 q-grid, N_G in [1500, 6000], N_v = 96, N_c in
  [800, 2400], N_eig = 10% of N_G, 48 frequencies): the first 16 q-points in one
  plan with device-drawn inputs, against the FP64 path on the two smallest.
* The 1/8-size subsample of the 12,000-plane-wave q-point (N_G = 1500, N_v = 32,
  N_c = 256, N_eig = 150, 48 frequencies): mixed path against the oracle.
"""
import numpy as np
import pytest

import oracle.rpa_oracle as orc
from paper_2405_20258_gb300 import inputs
from tests.gpu_helpers import run_gpu

pytestmark = pytest.mark.gpu


def device_problem(qp, n_eig, n_freq):
    import torch
    from paper_2405_20258_gb300 import rpa
    dq = rpa.device_qpoint(qp, n_eig, n_freq)
    A = torch.empty((qp.n_vc, qp.n_g), dtype=torch.complex128, device="cuda")
    rpa.rpa_generate_m(dq, 0, qp.n_v, 0, qp.n_c, A)
    torch.cuda.synchronize()
    dq.m = A
    return dq


def test_subspace_sizes_at_400_plane_waves():
    qp = inputs.make_qpoint(400, 16, 200)
    A = inputs.matrix_elements(qp)
    ref = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 200, 32)["ec"]
    got = run_gpu(qp, A, 200, 32, precision=1, keep=False)["ec"]
    assert abs(got - ref) <= 1e-6


def test_subspace_sizes_at_4000_plane_waves():
    from paper_2405_20258_gb300 import rpa
    qp = inputs.make_qpoint(4000, 128, 2000)
    errs = {}
    for n_eig in (200, 400, 800):
        dq = device_problem(qp, n_eig, 32)
        with rpa.Plan([dq], precision=rpa.RPA_FP64) as p:
            e64 = p.run(0)
        with rpa.Plan([dq], precision=rpa.RPA_MIXED) as p:
            emx = p.run(0)
        errs[n_eig] = abs(emx - e64)
        del dq
    print("mixed vs FP64 |dE_c| (Ha) by N_eig:", errs)
    for n_eig, e in errs.items():
        assert e <= 1e-6, (n_eig, e)


def test_uneven_batch_of_qpoints():
    from paper_2405_20258_gb300 import rpa
    sizes = inputs.batched_workload()[:16]
    dqs = []
    for s in sizes:
        qp = inputs.make_qpoint(s["n_g"], s["n_v"], s["n_c"], iq=s["iq"],
                                q_twentieths=s["q_twentieths"])
        dqs.append(rpa.device_qpoint(qp, max(1, s["n_g"] // 10), 48))  # A drawn on the device
    with rpa.Plan(dqs, precision=rpa.RPA_MIXED) as p:
        ecs = p.ecorr(-1)
    assert all(np.isfinite(ecs)) and all(e < 0 for e in ecs)
    # every q-point against the FP64 path (its own plan: FP64 contractions)
    with rpa.Plan(dqs, precision=rpa.RPA_FP64) as p:
        e64 = p.ecorr(-1)
    errs = [abs(a - b) for a, b in zip(ecs, e64)]
    print("uneven batch, mixed vs FP64 |dE_c| (Ha) per q-point:", errs)
    for i, e in enumerate(errs):
        assert e <= 1e-6, (i, ecs[i], e64[i])


def test_large_qpoint_subsample_against_oracle():
    qp = inputs.make_qpoint(1500, 32, 256)
    A = inputs.matrix_elements(qp)
    ref = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 150, 48)["ec"]
    got = run_gpu(qp, A, 150, 48, precision=1, keep=False)["ec"]
    assert abs(got - ref) <= 1e-6


def test_uneven_batch_smallest_qpoints_against_oracle():
    """The two smallest q-points of the uneven 64-q grid (by N_G N_vc), each in a plan of
    its own on the mixed path, against the oracle within 1e-6 Ha."""
    from paper_2405_20258_gb300 import rpa
    sizes = inputs.batched_workload()
    small = sorted(range(len(sizes)), key=lambda i: sizes[i]["n_g"] ** 2 * sizes[i]["n_c"])[:2]
    for i in small:
        s = sizes[i]
        qp = inputs.make_qpoint(s["n_g"], s["n_v"], s["n_c"], iq=s["iq"],
                                q_twentieths=s["q_twentieths"])
        A = inputs.matrix_elements(qp)
        n_eig = max(1, s["n_g"] // 10)
        ref = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, n_eig, 48)["ec"]
        got = run_gpu(qp, A, n_eig, 48, precision=1, keep=False)["ec"]
        assert abs(got - ref) <= 1e-6, (i, got, ref)
