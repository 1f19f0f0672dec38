"""Pins of the oracle's extensions: partial occupations and k-point weights
(the pair weight g_k (f_v - f_c) of Eq. chi0_partial_occs) and the slab-truncated
Coulomb kernel.  Each compares with an invariant, a closed form, or a numerical
integral, never with a re-typed oracle formula."""
import math

import numpy as np
import pytest

import oracle.rpa_oracle as orc
from paper_2405_20258_gb300 import inputs


def problem(n_g=12, n_v=2, n_c=4, n_k=1, seed=21):
    qp = inputs.make_qpoint(n_g, n_v, n_c, seed=seed, n_k=n_k)
    return qp, inputs.matrix_elements(qp)


def test_integer_occupations_one_kpoint_are_unweighted():
    qp, A = problem()
    ow = orc.pair_weights(np.ones(qp.n_v), np.zeros(qp.n_c))
    assert np.array_equal(ow, np.ones(qp.n_vc))
    a = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 6, 5)["ec"]
    b = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 6, 5, ow=ow)["ec"]
    assert a == b


def test_equal_occupation_pairs_drop_out():
    # the paper: pairs with f_n = f_n' contribute nothing (both occupied or both empty)
    qp, A = problem(n_v=2, n_c=3)
    occ_v = np.array([1.0, 0.5])
    occ_c = np.array([0.5, 0.0, 0.25])
    ow = orc.pair_weights(occ_v, occ_c)
    zero = np.where(ow == 0)[0]
    assert len(zero) == 1  # (v=1, c=0)
    keep = np.where(ow != 0)[0]
    delta = orc.transition_energies(qp.e_v, qp.e_c)
    for om in (0.0, 0.4):
        full = orc.chi0(A, delta, om, qp.omega_cell, ow)
        red = orc.chi0(A[keep], delta[keep], om, qp.omega_cell, ow[keep])
        assert np.max(np.abs(full - red)) < 1e-15 * np.max(np.abs(full))


def test_half_occupation_halves_chi0():
    qp, A = problem()
    delta = orc.transition_energies(qp.e_v, qp.e_c)
    ow = orc.pair_weights(np.full(qp.n_v, 0.75), np.full(qp.n_c, 0.25))
    assert np.allclose(ow, 0.5, rtol=0, atol=0)
    a = orc.chi0(A, delta, 0.3, qp.omega_cell, ow)
    b = orc.chi0(A, delta, 0.3, qp.omega_cell)
    assert np.max(np.abs(a - 0.5 * b)) < 1e-16 * np.max(np.abs(b))


def test_two_identical_kpoints_with_half_weights_equal_one():
    qp1, A1 = problem(n_k=1)
    e_v2 = np.stack([qp1.e_v, qp1.e_v])
    e_c2 = np.stack([qp1.e_c, qp1.e_c])
    A2 = np.concatenate([A1, A1])
    ow2 = orc.pair_weights(np.ones((2, qp1.n_v)), np.zeros((2, qp1.n_c)), [0.5, 0.5])
    d1 = orc.transition_energies(qp1.e_v, qp1.e_c)
    d2 = orc.transition_energies(e_v2, e_c2)
    assert np.array_equal(d2, np.concatenate([d1, d1]))
    x1 = orc.chi_tilde(A1, qp1.qg2, d1, 0.2, qp1.omega_cell)
    x2 = orc.chi_tilde(A2, qp1.qg2, d2, 0.2, qp1.omega_cell, ow2)
    assert np.max(np.abs(x1 - x2)) < 1e-14 * np.max(np.abs(x1))


def test_kpoint_row_order_matches_generator():
    qp, A = problem(n_v=2, n_c=3, n_k=2)
    assert A.shape == (2 * 2 * 3, qp.n_g)
    blk = inputs.matrix_elements(qp, v_range=[2, 3], c_range=[3, 4, 5])  # k = 1
    assert np.array_equal(A[6:], blk)
    d = orc.transition_energies(qp.e_v, qp.e_c)
    assert d[6 + 1 * 3 + 2] == qp.e_c[1, 2] - qp.e_v[1, 1]


def test_weighted_rank1_closed_form():
    qp, A = problem(n_g=7, n_v=1, n_c=1, seed=3)
    w = 0.37
    D = qp.e_c[0] - qp.e_v[0]
    s = float(np.sum(4 * math.pi / qp.qg2 * np.abs(A[0]) ** 2))
    alpha = 4 * s * w / qp.omega_cell
    out = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 1, 200, ow=np.array([w]))
    assert abs(out["ec"] - 0.5 * (math.sqrt(D * D + alpha * D) - D - alpha / 2)) < 1e-11 * abs(out["ec"])


@pytest.mark.parametrize("kpar,n", [(0.3, 0), (0.3, 1), (1.7, 2), (0.05, 3), (2.5, 5)])
def test_slab_coulomb_is_fourier_transform_of_truncated_potential(kpar, n):
    # 2-D transform of 1/r at fixed z is 2 pi exp(-k|z|)/k; integrate z over |z| < z_c
    from scipy.integrate import quad
    z_c = 5.0
    kz = math.pi * n / z_c   # (q+G)_z on the lattice of a cell of height 2 z_c
    val = 2 * quad(lambda z: 2 * math.pi / kpar * math.exp(-kpar * z), 0, z_c,
                   weight="cos", wvar=kz, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
    got = orc.coulomb_slab(np.array([[kpar, 0.0, kz]]), z_c)[0]
    assert abs(got - val) < 1e-11 * abs(val)


def test_slab_coulomb_limits():
    qp, _ = problem(n_g=30)
    k = inputs.qg_vectors(qp)
    assert np.allclose(np.sum(k * k, axis=1), qp.qg2, rtol=1e-14, atol=0)
    vs = orc.coulomb_slab(k, 5.0)
    vb = orc.coulomb(qp.qg2)
    assert np.all(vs > 0) and np.all(vs <= 2 * vb)
    # far from the slab (z_c much larger than 1/|q+G|_par, which is at most ~32 bohr) v is bare
    assert np.allclose(orc.coulomb_slab(k, 2000.0), vb, rtol=1e-12, atol=0)


def test_extensions_full_basis_equivalence_and_sign():
    qp, A = problem(n_g=14, n_v=2, n_c=3, n_k=2)
    occ_v = inputs.fermi_occupations(qp.e_v, 0.03, 0.02)
    occ_c = inputs.fermi_occupations(qp.e_c, 0.03, 0.02)
    ow = orc.pair_weights(occ_v, occ_c, [0.25, 0.75])
    assert np.all(ow > 0) and np.all(ow < 1)
    vg = orc.coulomb_slab(inputs.qg_vectors(qp), qp.a / 2)
    sub = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, qp.n_g, 8, ow=ow, vg=vg)["ec"]
    full = orc.ecorr_full_basis(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 8, ow=ow, vg=vg)
    assert sub < 0 and abs(sub - full) < 1e-11 * abs(full)
