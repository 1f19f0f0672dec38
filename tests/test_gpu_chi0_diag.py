"""GPU parity of the mixed path's FP64 chi~(0) diagonal (on by default;
RPA_TC_CHI0_DIAG=0 turns it off).

The digit-sliced GEMM multiplies only digit pairs s + t <= S - 1; on the diagonal
of chi~ = X^H X the dropped pairs include |d_s|^2 terms of one sign, so their
omission is a bias that adds up over the transitions.  Recomputing the diagonal
in FP64 removes it: measured at N_G = 4000, N_eig = 400, |dE_c| against the FP64
path falls from 1.8e-7 Ha to 2.1e-8 Ha with 4 slices.  Checked here: the
diagonal against the oracle's and E_c against the oracle at N_G = 400 (complex128
and complex64 inputs), and E_c against the FP64 path at N_G = 4000 with 3 and 4
slices.
"""
import numpy as np
import pytest

import oracle.rpa_oracle as orc
from paper_2405_20258_gb300 import inputs
from tests.gpu_helpers import run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [np.complex128, np.complex64])
def test_chi0_diagonal_matches_oracle_400(dtype):
    # complex64 A is read as given (its values widened exactly), so the oracle
    # takes the same rounded values in complex128
    qp = inputs.make_qpoint(400, 16, 200)
    A_in = inputs.matrix_elements(qp, dtype=dtype)
    A = A_in.astype(np.complex128)
    delta = orc.transition_energies(qp.e_v, qp.e_c)
    chit = orc.chi_tilde(A, qp.qg2, delta, 0.0, qp.omega_cell)
    mx = run_gpu(qp, A_in, 40, 16, precision=1)
    d_ref = np.real(np.diag(chit))
    assert np.max(np.abs(np.diag(mx["chit"]) - d_ref) / np.abs(d_ref)) < 1e-13
    assert np.max(np.abs(np.imag(np.diag(mx["chit"])))) == 0.0
    ref = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 40, 16)["ec"]
    assert abs(mx["ec"] - ref) <= 1e-6


def test_chi0_diagonal_off_switch(monkeypatch):
    # RPA_TC_CHI0_DIAG=0 keeps the sliced GEMM's diagonal: with 7 slices it still
    # agrees with the oracle's to the slicing's accuracy
    monkeypatch.setenv("RPA_TC_CHI0_DIAG", "0")
    qp = inputs.make_qpoint(200, 6, 50)
    A = inputs.matrix_elements(qp)
    delta = orc.transition_energies(qp.e_v, qp.e_c)
    chit = orc.chi_tilde(A, qp.qg2, delta, 0.0, qp.omega_cell)
    mx = run_gpu(qp, A, 20, 4, precision=1, slices=(7, 7, 7))
    d_ref = np.real(np.diag(chit))
    assert np.max(np.abs(np.diag(mx["chit"]) - d_ref) / np.abs(d_ref)) < 1e-12


@pytest.mark.parametrize("slices,tol", [((4, 6, 3), 1e-7), ((3, 6, 3), 6e-7)])
def test_chi0_diagonal_energy_4000(slices, tol):
    qp = inputs.make_qpoint(4000, 128, 2000)
    f64 = run_gpu(qp, None, 400, 32, precision=0, keep=False, generate=True)
    mx = run_gpu(qp, None, 400, 32, precision=1, keep=False, generate=True, slices=slices)
    assert abs(mx["ec"] - f64["ec"]) <= tol, mx["ec"] - f64["ec"]
