"""Parity of the mixed-precision (tcgen05, exact digit-sliced BF16) path.

* With 7 digit slices per operand the slicing error (about 2^-55 of the row
  scales) is below FP64 rounding, so the mixed path must reproduce the FP64
  CUDA path to FP64 accuracy: this pins the TMA/MMA/TMEM machinery exactly.
* With the default slices (4, 6, 3) the error is set by the digit truncation;
  at the 400-plane-wave workload it must stay within 1e-6 Ha of the oracle.
* Errors fall monotonically as slices are added.
* A stalled producer (test hook) makes every bounded wait run out: the stage
  reports RPA_ETIMEOUT and the context stays usable.
"""
import numpy as np
import pytest

import oracle.rpa_oracle as orc
from paper_2405_20258_gb300 import inputs
from tests.gpu_helpers import phases, rel_fro, run_gpu

pytestmark = pytest.mark.gpu


def problem(n_g, n_v, n_c, seed=inputs.DEFAULT_SEED):
    qp = inputs.make_qpoint(n_g, n_v, n_c, seed=seed)
    return qp, inputs.matrix_elements(qp)


def compare_exact(qp, A, n_eig, n_freq):
    f64 = run_gpu(qp, A, n_eig, n_freq, precision=0)
    mx = run_gpu(qp, A, n_eig, n_freq, precision=1, slices=(7, 7, 7))
    assert rel_fro(mx["chit"], f64["chit"]) < 1e-13
    assert np.max(np.abs(mx["lam0"] - f64["lam0"])) < 1e-13 * np.max(np.abs(f64["lam0"]))
    ph = phases(f64["C"], mx["C"])
    assert rel_fro(mx["Mt"] * ph[:, None], f64["Mt"]) < 1e-11
    al = ph[None, :, None] * np.conj(ph)[None, None, :]
    assert rel_fro(mx["chis"] * al, f64["chis"]) < 1e-11
    assert np.max(np.abs(mx["trace_k"] - f64["trace_k"]) / np.abs(f64["trace_k"])) < 1e-13
    assert abs(mx["ec"] - f64["ec"]) < 1e-12 * abs(f64["ec"])
    return f64, mx


def test_seven_slices_reproduce_fp64_ragged():
    qp, A = problem(150, 5, 37)
    compare_exact(qp, A, 23, 6)


@pytest.mark.parametrize("n_g,n_v,n_c,n_eig,n_freq", [(1, 2, 3, 1, 4), (40, 1, 1, 1, 3), (70, 2, 9, 1, 1),
                                                      (129, 3, 22, 129, 2), (200, 4, 70, 65, 9)])
def test_seven_slices_edge_shapes(n_g, n_v, n_c, n_eig, n_freq):
    qp, A = problem(n_g, n_v, n_c)
    compare_exact(qp, A, n_eig, n_freq)


def test_default_slices_within_1e6_of_oracle():
    """N_G=400, N_v=16, N_c=200, 16 frequencies: N_eig = 40 and N_eig = N_G."""
    qp, A = problem(400, 16, 200)
    for n_eig in (40, 400):
        ref = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, n_eig, 16)
        mx = run_gpu(qp, A, n_eig, 16, precision=1, keep=False)
        assert abs(mx["ec"] - ref["ec"]) <= 1e-6, (n_eig, mx["ec"] - ref["ec"])


def test_error_falls_with_slices():
    qp, A = problem(180, 4, 40)
    f64 = run_gpu(qp, A, 30, 4, precision=0)
    errs = []
    for s in (1, 2, 3, 4, 5):
        mx = run_gpu(qp, A, 30, 4, precision=1, slices=(s, s, s))
        errs.append(rel_fro(mx["chit"], f64["chit"]))
    for a, b in zip(errs, errs[1:]):
        assert b < a, errs
    # the truncation error of S digits is about 2^-(7 + 8(S-1)) of the row scales
    assert errs[2] < 2.0 ** -20 and errs[4] < 2.0 ** -36, errs


def test_complex64_input_mixed():
    qp = inputs.make_qpoint(120, 3, 30)
    A = inputs.matrix_elements(qp, dtype=np.complex64)
    ref = orc.ecorr(A.astype(np.complex128), qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 20, 4)
    mx = run_gpu(qp, A, 20, 4, precision=1, keep=False, slices=(7, 7, 7))
    assert abs(mx["ec"] - ref["ec"]) < 1e-11 * abs(ref["ec"])


def test_cholesky_route_mixed():
    qp, A = problem(160, 4, 30)
    ref = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 40, 6)
    mx = run_gpu(qp, A, 40, 6, precision=1, route="cholesky", keep=False, slices=(7, 7, 7))
    assert abs(mx["ec"] - ref["ec"]) < 1e-11 * abs(ref["ec"])


def test_bounded_wait_reports_timeout():
    import torch
    from paper_2405_20258_gb300 import rpa
    qp, A = problem(64, 2, 16)
    dq = rpa.device_qpoint(qp, 8, 2, A=A)
    with rpa.Plan([dq], precision=rpa.RPA_MIXED, debug_stall=1) as plan:
        plan.chi0_static(0)
        with pytest.raises(rpa.RPAError) as e:
            plan.subspace_basis(0)
        assert e.value.status == rpa.RPA_ETIMEOUT
    torch.cuda.synchronize()
    # the context is still healthy: a normal plan runs and matches the oracle
    ref = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 8, 2)["ec"]
    with rpa.Plan([rpa.device_qpoint(qp, 8, 2, A=A)], precision=rpa.RPA_MIXED,
                  slices=(7, 7, 7)) as plan:
        assert abs(plan.run(0) - ref) < 1e-11 * abs(ref)


@pytest.mark.parametrize("env", [
    {"RPA_TC_LE_CHI0": "5", "RPA_TC_LE_CHIS": "4"},   # every level exact, no tail
    {"RPA_TC_CHIS_OVERLAP": "0"},                      # chi_s planes cut on the plan stream
    {"RPA_TC_CHIS_GROUP": "1"},                        # one frequency per group: buffer reuse
    {"RPA_TC_BN": "64"},                               # narrow tiles everywhere
    {"RPA_TC_NA": "3", "RPA_TC_NB": "3", "RPA_TC_NACC": "1"},  # other pipeline depths
    {"RPA_TC_PROJ_CHUNK": "128"},                      # projection in chunks of 128 rows of A
])
def test_gemm_variants_agree(env, monkeypatch):
    """Tail accumulator, side-stream cutting, tile width, pipeline depth and the
    projection's row chunks are implementation choices: every variant gives the
    default's E_c and chi~ to within the digit truncation of (5, 6, 4) slices."""
    qp, A = problem(200, 4, 50)
    base = run_gpu(qp, A, 40, 6, precision=1, slices=(5, 6, 4))
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    got = run_gpu(qp, A, 40, 6, precision=1, slices=(5, 6, 4))
    assert rel_fro(got["chit"], base["chit"]) < 1e-10
    assert abs(got["ec"] - base["ec"]) < 1e-10 * abs(base["ec"])


def test_interleaved_stages_of_two_qpoints():
    """The plan holds one q-point's intermediates per stage.  Interleaving the
    stages of two q-points gives their one-after-the-other energies while each
    stage still finds its predecessor's outputs (the projection planes cut during
    one q-point's eigensolve being replaced by the other's chi~ blocks on the way);
    a stage whose inputs another q-point has replaced returns RPA_ESTATE."""
    import torch
    from paper_2405_20258_gb300 import rpa
    qa = inputs.make_qpoint(160, 3, 40, iq=0)
    qb = inputs.make_qpoint(130, 4, 30, iq=1, seed=inputs.DEFAULT_SEED + 7)
    dqs = [rpa.device_qpoint(q, 30, 6, A=inputs.matrix_elements(q)) for q in (qa, qb)]
    with rpa.Plan(dqs, precision=rpa.RPA_MIXED) as p:
        seq = [p.run(0), p.run(1)]
        p.chi0_static(0)
        p.subspace_basis(0)      # cuts q-point 0's projection planes on the side stream
        p.chi0_static(1)         # chi~ of q-point 1 (its K-blocks replace those planes)
        p.chi_freq(0)            # q-point 0's basis is still held
        e0 = p.ecorr(0)
        p.subspace_basis(1)
        p.chi_freq(1)
        e1 = p.ecorr(1)
        torch.cuda.synchronize()
        for a, b in zip(seq, (e0, e1)):
            assert abs(a - b) <= 1e-12 * abs(a), (seq, (e0, e1))
        p.chi0_static(0)
        p.chi0_static(1)         # replaces q-point 0's chi~
        with pytest.raises(rpa.RPAError) as e:
            p.subspace_basis(0)
        assert e.value.status == rpa.RPA_ESTATE
        with pytest.raises(rpa.RPAError) as e:
            p.ecorr(0)           # chi_s held is q-point 1's
        assert e.value.status == rpa.RPA_ESTATE
        p.subspace_basis(1)
        p.chi_freq(1)
        assert abs(p.ecorr(1) - seq[1]) <= 1e-12 * abs(seq[1])
