"""GPU parity of the extensions: partial occupations and several k-points
(pair weights g_k (f_v - f_c) of Eq. chi0_partial_occs) and the slab-truncated
Coulomb kernel, on the FP64 path against the oracle and on the mixed path (7
digit slices) against the FP64 path."""
import numpy as np
import pytest

import oracle.rpa_oracle as orc
from paper_2405_20258_gb300 import inputs
from tests.gpu_helpers import rel_fro, run_gpu

pytestmark = pytest.mark.gpu


def ext_problem(n_g, n_v, n_c, n_k=1, occ=True, slab=True, seed=inputs.DEFAULT_SEED):
    qp = inputs.make_qpoint(n_g, n_v, n_c, n_k=n_k, seed=seed)
    A = inputs.matrix_elements(qp)
    extra, ow, vg = {}, None, None
    occ_v = occ_c = None
    if occ:
        occ_v = inputs.fermi_occupations(qp.e_v, 0.03, 0.15)
        occ_c = inputs.fermi_occupations(qp.e_c, 0.03, 0.15)
        extra.update(occ_v=occ_v, occ_c=occ_c)
    kw = None
    if n_k > 1:
        kw = np.linspace(1.0, 2.0, n_k)
        kw /= kw.sum()
        extra.update(k_weight=kw)
    if occ or n_k > 1:
        ow = orc.pair_weights(occ_v if occ_v is not None else np.ones((n_k, n_v)),
                              occ_c if occ_c is not None else np.zeros((n_k, n_c)), kw)
    if slab:
        qv = inputs.qg_vectors(qp)
        vg = orc.coulomb_slab(qv, qp.a / 2)
        extra.update(slab_zc=qp.a / 2, qg_vec=qv)
    return qp, A, ow, vg, extra


def check(qp, A, ow, vg, extra, n_eig, n_freq):
    ref = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, n_eig, n_freq, keep=True, ow=ow, vg=vg)
    got = run_gpu(qp, A, n_eig, n_freq, **extra)
    assert rel_fro(got["chit"], ref["chit"]) < 1e-12
    assert np.max(np.abs(got["lam0"] - ref["lam0"])) < 1e-12 * np.max(np.abs(ref["lam0"]))
    assert np.max(np.abs(got["trace_k"] - ref["trace_k"]) / np.abs(ref["trace_k"])) < 1e-12
    lsc = np.max(np.abs(ref["lam_k"]))
    assert np.max(np.abs(np.sort(got["lam_k"], axis=1) - ref["lam_k"])) < 1e-11 * lsc
    assert abs(got["ec"] - ref["ec"]) <= 1e-8
    return ref, got


def test_partial_occupations():
    qp, A, ow, vg, extra = ext_problem(110, 4, 30, occ=True, slab=False)
    assert np.all(ow > 0) and np.any(ow < 0.9)
    check(qp, A, ow, vg, extra, 25, 6)


def test_two_kpoints_with_weights():
    qp, A, ow, vg, extra = ext_problem(90, 3, 20, n_k=2, occ=False, slab=False)
    check(qp, A, ow, vg, extra, 30, 5)


def test_slab_coulomb():
    qp, A, ow, vg, extra = ext_problem(130, 3, 25, occ=False, slab=True)
    check(qp, A, ow, vg, extra, 20, 6)


def test_all_extensions_fp64_and_mixed():
    qp, A, ow, vg, extra = ext_problem(150, 3, 22, n_k=3, occ=True, slab=True)
    ref, f64 = check(qp, A, ow, vg, extra, 40, 7)
    mx = run_gpu(qp, A, 40, 7, precision=1, slices=(7, 7, 7), **extra)
    assert rel_fro(mx["chit"], f64["chit"]) < 1e-13
    assert abs(mx["ec"] - f64["ec"]) < 1e-12 * abs(f64["ec"])
    dflt = run_gpu(qp, A, 40, 7, precision=1, keep=False, **extra)
    assert abs(dflt["ec"] - ref["ec"]) < 1e-6


def test_generated_kpoints_match_host_generator():
    qp, A, ow, vg, extra = ext_problem(70, 2, 15, n_k=2, occ=True, slab=False)
    ref = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 20, 4, ow=ow)["ec"]
    got = run_gpu(qp, A, 20, 4, keep=False, generate=True, **extra)
    assert abs(got["ec"] - ref) <= 1e-8


def test_pair_weight_of_wrong_sign_is_rejected():
    from paper_2405_20258_gb300 import rpa
    qp, A, ow, vg, extra = ext_problem(40, 2, 6, occ=False, slab=False)
    occ_v = np.zeros(qp.n_v)      # empty valence, full conduction: w < 0 with Delta > 0
    occ_c = np.ones(qp.n_c)
    with pytest.raises(rpa.RPAError) as e:
        run_gpu(qp, A, 5, 2, occ_v=occ_v, occ_c=occ_c)
    assert e.value.status == rpa.RPA_EINVAL and "pair weights" in str(e.value)
