"""GPU parity of the library's own subspace eigensolver of chi~(0) (step a3).

Every plan takes it by default: FP64 plans (and mixed plans below N_G = 1024)
start from an FP64 Householder reduction, mixed plans from N_G = 1024 on from
the FP32 reduction of chi~/max|chi~| followed by a degree-3 Chebyshev filter.
Both then orthonormalise by Cholesky-QR2 and take a Rayleigh-Ritz step whose
small eigenproblem is solved by Jacobi rotations in FP64.  The FP64 start is
checked element by element against the oracle in test_gpu_fp64.py; here:

* the FP32 start at N_G = 1024 (eigenvalues and the largest principal-angle sine of
  the subspace against LAPACK on the chi~ the solver was given, E_c within 1e-7 Ha
  of the oracle), with the block products on the tensor cores or the FP64 pipe and
  with one or two filter steps;
* Jacobi's eigenvectors orthonormal to FP64 rounding (C^H C = I);
* the library solver, kept as the fallback for degenerate spectra
  (RPA_EIG=cusolver), against the own solver.
"""
import numpy as np
import pytest

import oracle.rpa_oracle as orc
from paper_2405_20258_gb300 import inputs
from tests.gpu_helpers import run_gpu

pytestmark = pytest.mark.gpu


def sin_angle(U, V):
    Qu, _ = np.linalg.qr(U)
    Qv, _ = np.linalg.qr(V)
    return np.linalg.norm(Qv - Qu @ (Qu.conj().T @ Qv), 2)


@pytest.fixture(scope="module")
def problem_1024():
    qp = inputs.make_qpoint(1024, 32, 1000)
    A = inputs.matrix_elements(qp)
    n_eig, n_freq = 128, 16
    ref = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, n_eig, n_freq, keep=True)
    delta = orc.transition_energies(qp.e_v, qp.e_c)
    chit = orc.chi_tilde(A, qp.qg2, delta, 0.0, qp.omega_cell)
    _, V = np.linalg.eigh(chit)
    return qp, A, n_eig, n_freq, ref, V[:, :n_eig]


@pytest.mark.parametrize("tc,steps", [("1", "1"), ("0", "1"), ("1", "2")])
def test_fp32_start_vs_oracle_1024(monkeypatch, problem_1024, tc, steps):
    qp, A, n_eig, n_freq, ref, V = problem_1024
    monkeypatch.setenv("RPA_EIG_TC", tc)
    monkeypatch.setenv("RPA_EIG_STEPS", steps)
    mx = run_gpu(qp, A, n_eig, n_freq, precision=1)
    # the eigensolver against LAPACK on the chi~ it was given (the sliced chi~ of the
    # mixed path), the whole path against the oracle through E_c
    w_own, v_own = np.linalg.eigh(mx["chit"])
    lam_ref = w_own[:n_eig]
    err_lam = np.max(np.abs(mx["lam0"] - lam_ref)) / np.max(np.abs(lam_ref))
    sine = sin_angle(mx["C"], v_own[:, :n_eig])
    orth = np.max(np.abs(mx["C"].conj().T @ mx["C"] - np.eye(n_eig)))
    print("FP32 start tc=%s steps=%s: eigenvalues %.2e, sine %.2e, orth %.2e, dE_c %.2e, "
          "sine to the oracle's subspace %.2e" % (tc, steps, err_lam, sine, orth,
                                                   mx["ec"] - ref["ec"], sin_angle(mx["C"], V)))
    assert err_lam < 1e-12
    assert sine < 5e-8
    assert orth < 1e-13
    assert abs(mx["ec"] - ref["ec"]) <= 1e-7, mx["ec"] - ref["ec"]


def test_fp64_start_in_a_mixed_plan_vs_oracle_1024(monkeypatch, problem_1024):
    qp, A, n_eig, n_freq, ref, V = problem_1024
    monkeypatch.setenv("RPA_EIG_START32", "0")
    mx = run_gpu(qp, A, n_eig, n_freq, precision=1)
    # against LAPACK on the sliced chi~ the solver was given; E_c against the oracle
    w_own, v_own = np.linalg.eigh(mx["chit"])
    assert np.max(np.abs(mx["lam0"] - w_own[:n_eig])) < 1e-12 * np.max(np.abs(w_own))
    # LAPACK's own subspace is resolved to ~eps |H| / gap at the cut (~2e-8 here)
    assert sin_angle(mx["C"], v_own[:, :n_eig]) < 5e-8
    assert abs(mx["ec"] - ref["ec"]) <= 1e-7


@pytest.mark.parametrize("precision", [0, 1])
def test_library_fallback_agrees(monkeypatch, precision):
    qp = inputs.make_qpoint(300, 8, 60)
    A = inputs.matrix_elements(qp)
    own = run_gpu(qp, A, 50, 8, precision=precision)
    monkeypatch.setenv("RPA_EIG", "cusolver")
    lib = run_gpu(qp, A, 50, 8, precision=precision)
    P_own = own["C"] @ own["C"].conj().T
    P_lib = lib["C"] @ lib["C"].conj().T
    assert np.max(np.abs(P_own - P_lib)) < 1e-9
    assert abs(own["ec"] - lib["ec"]) <= 1e-8


def test_basis_orthonormal_fp64_full_subspace():
    qp = inputs.make_qpoint(400, 16, 200)
    A = inputs.matrix_elements(qp)
    got = run_gpu(qp, A, 400, 4)
    C = got["C"]
    assert np.max(np.abs(C.conj().T @ C - np.eye(400))) < 1e-13
