"""Parity of the FP64 CUDA path with the FP64 oracle, stage by stage.

Sizes span several 64-wide tiles with ragged tails; edge cases cover
N_eig = 1, N_eig = N_G, a single transition, a single plane wave and one
frequency.  Tolerances: relative Frobenius error <= 1e-12 for chi~ and chi_s,
|dE_c| <= 1e-8 Ha on the FP64 path.
"""
import math

import numpy as np
import pytest

import oracle.rpa_oracle as orc
from paper_2405_20258_gb300 import inputs
from tests.gpu_helpers import phases, rel_fro, run_gpu

pytestmark = pytest.mark.gpu


def problem(n_g, n_v, n_c, seed=inputs.DEFAULT_SEED, dtype=np.complex128):
    qp = inputs.make_qpoint(n_g, n_v, n_c, seed=seed)
    return qp, inputs.matrix_elements(qp, dtype=dtype)


def compare_all(qp, A, n_eig, n_freq, ec_abs=1e-8, route="eig"):
    ref = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, n_eig, n_freq, keep=True)
    got = run_gpu(qp, A, n_eig, n_freq, route=route)
    # quadrature
    assert np.max(np.abs(got["omega"] - ref["omega"]) / ref["omega"]) < 1e-12
    assert np.max(np.abs(got["weight"] - ref["weight"]) / ref["weight"]) < 1e-12
    # chi~(0): Hermitian, matches element by element
    assert rel_fro(got["chit"], ref["chit"]) < 1e-12
    assert np.max(np.abs(got["chit"] - ref["chit"])) < 1e-12 * np.max(np.abs(ref["chit"]))
    assert np.array_equal(got["chit"], got["chit"].conj().T)
    # eigenvalues and eigenvectors (up to a phase per column)
    scale = np.max(np.abs(ref["lam0"]))
    assert np.max(np.abs(got["lam0"] - ref["lam0"])) < 1e-12 * scale
    # the subspace itself (projector C C^H) is unique
    P_ref = ref["C"] @ ref["C"].conj().T
    P_gpu = got["C"] @ got["C"].conj().T
    assert np.max(np.abs(P_gpu - P_ref)) < 1e-9
    # gauge pivots real positive
    piv = got["C"][np.argmax(np.abs(got["C"]), axis=0), np.arange(n_eig)]
    assert np.all(piv.imag == 0) and np.all(piv.real > 0)
    # individual eigenvectors, M~ rows and chi_s entries are unique (up to the
    # phase) only for well separated eigenvalues: compare those after aligning
    lam_all = ref["lam_all"]
    d = np.diff(lam_all)
    sep = np.minimum(np.r_[np.inf, d][:n_eig], np.r_[d, np.inf][:n_eig]) / max(scale, 1e-300)
    ok = sep > 1e-7
    ph = phases(ref["C"], got["C"])
    assert np.max(np.abs((got["C"] * np.conj(ph) - ref["C"])[:, ok]), initial=0) < 1e-8
    assert rel_fro((got["Mt"] * ph[:, None])[ok], ref["Mt"][ok]) < 1e-9 if ok.any() else True
    al = ph[None, :, None] * np.conj(ph)[None, None, :]
    sel = np.ix_(np.arange(n_freq), np.where(ok)[0], np.where(ok)[0])
    if ok.any():
        assert rel_fro((got["chis"] * al)[sel], ref["chis"][sel]) < 1e-9
    # Frobenius norm of each chi_s is gauge invariant
    for k in range(n_freq):
        assert abs(np.linalg.norm(got["chis"][k]) / np.linalg.norm(ref["chis"][k]) - 1) < 1e-12
    # gauge-invariant quantities
    assert np.max(np.abs(got["trace_k"] - ref["trace_k"]) / np.abs(ref["trace_k"])) < 1e-12
    if route == "eig":
        lsc = np.max(np.abs(ref["lam_k"]))
        assert np.max(np.abs(np.sort(got["lam_k"], axis=1) - ref["lam_k"])) < 1e-11 * lsc
    assert abs(got["ec"] - ref["ec"]) <= ec_abs, (got["ec"], ref["ec"])
    return ref, got


def test_small_ragged_tiles():
    qp, A = problem(150, 5, 37)
    compare_all(qp, A, 23, 6)


def test_full_basis_neig_equals_ng():
    qp, A = problem(97, 3, 20)
    ref, got = compare_all(qp, A, 97, 5)
    full = orc.ecorr_full_basis(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 5)
    assert abs(got["ec"] - full) < 1e-11 * abs(full)


def test_single_transition_closed_form():
    qp, A = problem(9, 1, 1, seed=3)
    got = run_gpu(qp, A, 1, 12)
    D = qp.e_c[0] - qp.e_v[0]
    s = float(np.sum(4 * math.pi / qp.qg2 * np.abs(A[0]) ** 2))
    alpha = 4 * s / qp.omega_cell
    lam = -alpha * D / (D * D + got["omega"] ** 2)
    assert np.max(np.abs(got["lam_k"][:, 0] - lam)) < 1e-13 * np.max(np.abs(lam))
    e = np.sum(got["weight"] * (np.log1p(-lam) + lam)) / (2 * math.pi)
    assert abs(got["ec"] - e) < 1e-13 * abs(e)


@pytest.mark.parametrize("n_g,n_v,n_c,n_eig,n_freq", [(1, 2, 3, 1, 4), (40, 1, 1, 1, 3), (70, 2, 9, 1, 1),
                                                      (65, 2, 33, 65, 2), (128, 4, 16, 64, 7)])
def test_edge_shapes(n_g, n_v, n_c, n_eig, n_freq):
    qp, A = problem(n_g, n_v, n_c)
    compare_all(qp, A, n_eig, n_freq)


def test_complex64_input():
    qp, A = problem(90, 3, 30, dtype=np.complex64)
    ref = orc.ecorr(A.astype(np.complex128), qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 20, 4)
    got = run_gpu(qp, A, 20, 4, keep=False)
    assert abs(got["ec"] - ref["ec"]) <= 1e-8


def test_cholesky_route_matches_eigen_route():
    qp, A = problem(120, 4, 25)
    ref, got = compare_all(qp, A, 30, 6, route="cholesky")


def test_config1_sizes_both_subspaces():
    """N_G=400, N_v=16, N_c=200, 16 frequencies, N_eig = N_G and 40."""
    qp, A = problem(400, 16, 200)
    for n_eig in (400, 40):
        compare_all(qp, A, n_eig, 16)


def test_device_generator_matches_host():
    import torch
    from paper_2405_20258_gb300 import rpa
    qp = inputs.make_qpoint(77, 5, 11, iq=3)
    dq = rpa.device_qpoint(qp, 4, 2)
    for dt, tol in ((torch.complex128, 4e-15), (torch.complex64, 0.0)):
        out = torch.empty((3 * 4, 77), dtype=dt, device="cuda")
        rpa.rpa_generate_m(dq, 1, 3, 6, 4, out)
        host = inputs.matrix_elements(qp, v_range=range(1, 4), c_range=range(6, 10),
                                      dtype=np.complex128 if dt == torch.complex128 else np.complex64)
        d = out.cpu().numpy()
        err = np.max(np.abs(d - host) / np.abs(host))
        if tol == 0.0:
            # float rounding of the same double may differ by one float ulp
            assert err < 2 ** -23
        else:
            assert err < tol


def test_generated_matrix_path_matches_oracle():
    qp, A = problem(100, 4, 30)
    ref = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 25, 5)
    got = run_gpu(qp, A, 25, 5, keep=False, generate=True)
    assert abs(got["ec"] - ref["ec"]) <= 1e-8


def test_multi_qpoint_plan():
    import torch
    from paper_2405_20258_gb300 import rpa
    qs, refs, dqs = [], [], []
    for iq, (ng, nv, nc) in enumerate([(60, 2, 10), (130, 3, 7), (45, 1, 20)]):
        qp = inputs.make_qpoint(ng, nv, nc, iq=iq, q_twentieths=inputs.qgrid_4x4x4()[iq])
        A = inputs.matrix_elements(qp)
        refs.append(orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, ng // 3, 6)["ec"])
        dqs.append(rpa.device_qpoint(qp, ng // 3, 6, A=A))
    with rpa.Plan(dqs) as plan:
        ecs = plan.ecorr(-1)
    for e, r in zip(ecs, refs):
        assert abs(e - r) <= 1e-8


def test_errors_and_stage_order():
    import torch
    from paper_2405_20258_gb300 import rpa
    qp, A = problem(30, 2, 5)
    dq = rpa.device_qpoint(qp, 5, 3, A=A)
    with rpa.Plan([dq]) as plan:
        with pytest.raises(rpa.RPAError) as e:
            plan.subspace_basis(0)
        assert e.value.status == rpa.RPA_ESTATE
        with pytest.raises(rpa.RPAError) as e:
            plan.chi0_static(1)
        assert e.value.status == rpa.RPA_EINVAL
        # the plan is still usable after the errors
        ref = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 5, 3)["ec"]
        assert abs(plan.run(0) - ref) <= 1e-8
    # non-positive transition energy is rejected
    bad = rpa.device_qpoint(qp, 5, 3, A=A)
    bad.e_c = torch.full_like(bad.e_c, -1.0)
    with rpa.Plan([bad]) as plan:
        with pytest.raises(rpa.RPAError) as e:
            plan.chi0_static(0)
        assert e.value.status == rpa.RPA_EINVAL


@pytest.mark.parametrize("n_eig", [1, 31, 32, 33, 64, 97, 400])
def test_tiled_cholesky_route_config1(n_eig):
    """ln det(1 - chi_s) by the tiled Cholesky (32-wide tiles): one tile, a tile
    edge, ragged tails and the full 13-tile basis, against the oracle's E_c (its
    eigenvalues) at N_G = 400, 16 frequencies."""
    qp, A = problem(400, 16, 200)
    ref = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, n_eig, 16)
    got = run_gpu(qp, A, n_eig, 16, route="cholesky", keep=False)
    assert abs(got["ec"] - ref["ec"]) <= 1e-8, (got["ec"], ref["ec"])


def test_fp64_path_at_4000_plane_waves_vc_subsample():
    """The N_G = 4000 workload (N_c = 2000, N_eig = 400, 32 frequencies) with N_v
    subsampled to 4 of 128 so that the oracle finishes in seconds: chi~ to 1e-12
    relative Frobenius, the basis eigenvalues, and E_c to 1e-8 Ha."""
    qp, A = problem(4000, 4, 2000)
    ref = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 400, 32, keep=True)
    got = run_gpu(qp, A, 400, 32, route="cholesky")
    assert rel_fro(got["chit"], ref["chit"]) < 1e-12
    scale = np.max(np.abs(ref["lam0"]))
    assert np.max(np.abs(got["lam0"] - ref["lam0"])) < 1e-12 * scale
    assert np.max(np.abs(got["trace_k"] - ref["trace_k"]) / np.abs(ref["trace_k"])) < 1e-12
    assert abs(got["ec"] - ref["ec"]) <= 1e-8, (got["ec"], ref["ec"])
