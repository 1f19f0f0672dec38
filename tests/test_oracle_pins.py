"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these re-types an oracle formula: each compares the oracle with a
closed form, an invariant, a different algorithm (LU log-determinant,
Cholesky), brute-force loops on tiny inputs, or a textbook property of the
quadrature.  The mutation tests at the end plant a plausible mistake in the
oracle (on the CPU) and check that some pin catches it.
"""
import math

import numpy as np
import pytest

import oracle.rpa_oracle as orc
from paper_2405_20258_gb300 import inputs


def tiny_problem(n_g=6, n_v=2, n_c=3, seed=7):
    qp = inputs.make_qpoint(n_g, n_v, n_c, seed=seed)
    A = inputs.matrix_elements(qp)
    return qp, A


# --- quadrature (Computational Details: Gauss-Legendre on the imaginary axis) ---

@pytest.mark.parametrize("n", [1, 4, 16, 32, 48])
def test_quadrature_exact_for_polynomials(n):
    # with w = s t/(1-t), dw = s/(1-t)^2 dt, so weight*(1-t)^2/s is the plain GL
    # rule on [0,1]: it integrates t^m exactly for m <= 2n-1.
    s = 0.5
    om, wt = orc.frequency_grid(n, s)
    t = om / (s + om)
    for m in range(2 * n):
        got = np.sum(wt * (1 - t) ** 2 / s * t ** m)
        assert abs(got - 1.0 / (m + 1)) < 1e-13, (m, got)


def test_quadrature_integrates_lorentzian():
    # int_0^inf D/(D^2+w^2) dw = pi/2 for any D > 0
    om, wt = orc.frequency_grid(64, 0.5)
    for D in (0.1, 0.7, 3.0):
        got = np.sum(wt * D / (D * D + om * om))
        assert abs(got - math.pi / 2) < 1e-8


def test_quadrature_mapped_nodes_positive_and_ordered():
    om, wt = orc.frequency_grid(32, 0.5)
    assert np.all(om > 0) and np.all(np.diff(om) > 0) and np.all(wt > 0)


# --- chi0 (Eq. chi0_partial_occs) ---------------------------------------------

def test_chi0_bruteforce_loops():
    qp, A = tiny_problem(5, 2, 3)
    delta = orc.transition_energies(qp.e_v, qp.e_c)
    for omega in (0.0, 0.37):
        ref = np.zeros((qp.n_g, qp.n_g), complex)
        for v in range(qp.n_v):
            for c in range(qp.n_c):
                vc = v * qp.n_c + c
                d = qp.e_c[c] - qp.e_v[v]
                # resonant + anti-resonant terms of 2(f_c - f_v)/(e_c - e_v - i w), f_v=1, f_c=0
                wgt = (-2.0 / (d - 1j * omega) - 2.0 / (d + 1j * omega)).real
                for g in range(qp.n_g):
                    for h in range(qp.n_g):
                        ref[g, h] += np.conj(A[vc, g]) * wgt * A[vc, h] / qp.omega_cell
        got = orc.chi0(A, delta, omega, qp.omega_cell)
        assert np.max(np.abs(got - ref)) < 1e-14 * np.max(np.abs(ref))


def test_chi0_hermitian_negative_semidefinite():
    qp, A = tiny_problem(24, 3, 5)
    delta = orc.transition_energies(qp.e_v, qp.e_c)
    for omega in (0.0, 0.2, 5.0):
        x = orc.chi0(A, delta, omega, qp.omega_cell)
        assert np.max(np.abs(x - x.conj().T)) < 1e-15 * np.max(np.abs(x))
        lam = np.linalg.eigvalsh(x)
        assert lam.max() < 1e-13 * abs(lam.min())


def test_chi_tilde_trace_bruteforce():
    qp, A = tiny_problem(7, 2, 2)
    delta = orc.transition_energies(qp.e_v, qp.e_c)
    om = 0.3
    tot = 0.0
    for vc in range(A.shape[0]):
        f = 4 * delta[vc] / (delta[vc] ** 2 + om ** 2)
        for g in range(qp.n_g):
            tot -= f * (4 * math.pi / qp.qg2[g]) * abs(A[vc, g]) ** 2 / qp.omega_cell
    x = orc.chi_tilde(A, qp.qg2, delta, om, qp.omega_cell)
    assert abs(np.trace(x).real - tot) < 1e-13 * abs(tot)


# --- rank-1 closed form (Eq. rpaE with one transition) -----------------------

def rank1_problem(n_g=6, seed=3):
    qp, A = tiny_problem(n_g, 1, 1, seed)
    D = qp.e_c[0] - qp.e_v[0]
    s = float(np.sum(4 * math.pi / qp.qg2 * np.abs(A[0]) ** 2))
    alpha = 4 * s / qp.omega_cell
    return qp, A, D, alpha


def test_rank1_eigenvalue_per_node():
    qp, A, D, alpha = rank1_problem()
    out = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 1, 12, keep=True)
    om = out["omega"]
    lam_exact = -alpha * D / (D * D + om * om)
    assert np.max(np.abs(out["lam_k"][:, 0] - lam_exact)) < 1e-13 * abs(lam_exact).max()
    e_quad = np.sum(out["weight"] * (np.log1p(-lam_exact) + lam_exact)) / (2 * math.pi)
    assert abs(out["ec"] - e_quad) < 1e-13 * abs(e_quad)


def test_rank1_converges_to_closed_form():
    qp, A, D, alpha = rank1_problem()
    closed = 0.5 * (math.sqrt(D * D + alpha * D) - D - alpha / 2)
    errs = []
    for n in (8, 32, 200):
        e = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 1, n)["ec"]
        errs.append(abs(e - closed))
    assert errs[-1] < 1e-11 * abs(closed)
    assert errs[0] > errs[-1]


def test_rank1_closed_form_scipy_quad():
    # the closed form itself against adaptive quadrature of the integrand
    from scipy.integrate import quad
    for D, al in [(0.7, 3.3), (0.04, 0.5), (2.5, 40.0)]:
        f = lambda w: (math.log1p(al * D / (D * D + w * w)) - al * D / (D * D + w * w)) / (2 * math.pi)
        val = quad(f, 0, np.inf, epsabs=1e-14, epsrel=1e-13, limit=400)[0]
        assert abs(val - 0.5 * (math.sqrt(D * D + al * D) - D - al / 2)) < 1e-10


# --- subspace machinery (Method: C_s, M_s = M C_s, chi0_s = M_s^+ Delta M_s) --

def test_full_basis_equivalence_lu():
    qp, A = tiny_problem(14, 2, 5, seed=11)
    nf = 10
    sub = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, qp.n_g, nf)["ec"]
    full = orc.ecorr_full_basis(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, nf)
    assert sub < 0
    assert abs(sub - full) < 1e-11 * abs(full)


def test_chis_static_is_diagonal_lambda():
    qp, A = tiny_problem(20, 2, 6, seed=5)
    out = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 8, 4, keep=True)
    delta = orc.transition_energies(qp.e_v, qp.e_c)
    x0 = orc.chi_s(out["Mt"], delta, 0.0, qp.omega_cell)
    assert np.max(np.abs(x0 - np.diag(out["lam0"]))) < 1e-12 * abs(out["lam0"]).max()
    # the selected eigenvalues are the most negative ones
    assert np.all(out["lam0"] <= out["lam_all"][8] + 1e-15)


def test_sylvester_logdet_and_trace():
    qp, A = tiny_problem(16, 2, 4, seed=9)
    out = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, qp.n_g, 6, keep=True)
    delta = orc.transition_energies(qp.e_v, qp.e_c)
    for k in range(6):
        lam = out["lam_k"][k]
        ld_chol = orc.logdet_cholesky(out["chis"][k])
        full = orc.chi_tilde(A, qp.qg2, delta, out["omega"][k], qp.omega_cell)
        ld_lu = np.linalg.slogdet(np.eye(qp.n_g) - full)[1]
        assert abs(np.sum(np.log1p(-lam)) - ld_chol) < 1e-11 * abs(ld_lu)
        assert abs(ld_chol - ld_lu) < 1e-11 * abs(ld_lu)
        assert abs(out["trace_k"][k] - lam.sum()) < 1e-12 * abs(lam).sum()


def test_projection_bruteforce():
    qp, A = tiny_problem(6, 1, 3, seed=2)
    C = np.linalg.qr(np.random.default_rng(0).standard_normal((6, 3)) + 1j)[0]
    Mt = orc.project(A, qp.qg2, C)
    for i in range(3):
        for vc in range(A.shape[0]):
            s = sum(A[vc, g] * math.sqrt(4 * math.pi / qp.qg2[g]) * C[g, i] for g in range(6))
            assert abs(Mt[i, vc] - np.conj(s)) < 1e-13 * abs(s) + 1e-300


def test_gauge_invariance_and_canonical_phase():
    qp, A = tiny_problem(18, 2, 4, seed=4)
    delta = orc.transition_energies(qp.e_v, qp.e_c)
    chit = orc.chi_tilde(A, qp.qg2, delta, 0.0, qp.omega_cell)
    lam, C, _ = orc.subspace_basis(chit, 5)
    idx = np.argmax(np.abs(C), axis=0)
    piv = C[idx, np.arange(5)]
    assert np.all(np.abs(piv.imag) < 1e-15) and np.all(piv.real > 0)
    # E_c does not depend on the eigenvector phases
    ph = np.exp(1j * np.random.default_rng(1).uniform(0, 6.3, 5))
    Mt1 = orc.project(A, qp.qg2, C)
    Mt2 = orc.project(A, qp.qg2, C * ph[None, :])
    for om in (0.0, 0.9):
        l1 = np.linalg.eigvalsh(orc.chi_s(Mt1, delta, om, qp.omega_cell))
        l2 = np.linalg.eigvalsh(orc.chi_s(Mt2, delta, om, qp.omega_cell))
        assert np.max(np.abs(l1 - l2)) < 1e-12 * abs(l1).max()


def test_energy_negative_and_terms_nonpositive():
    qp, A = tiny_problem(30, 3, 6, seed=13)
    out = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 10, 8, keep=True)
    assert out["ec"] < 0
    assert np.all(out["lam_k"] <= 1e-12 * abs(out["lam_k"]).max())
    assert np.all(out["e_k"] <= 0)


def test_subspace_interlacing_bounds_and_monotone_energy():
    # chi_s(iw) = C^H chi~(iw) C is a compression of chi~(iw) = v^1/2 chi0(iw) v^1/2
    # onto orthonormal columns (Method: M_s = M C_s), so Cauchy interlacing holds:
    # lambda_i <= mu_i <= lambda_{i + N_G - N_eig} (ascending).  f(l) = ln(1-l) + l is
    # increasing and <= 0 for l <= 0, so every node's term, and E_c, can only rise
    # (towards 0) when the subspace shrinks, and equal the full-basis value at N_G.
    # This bounds the truncation error; its size has no closed form.
    qp, A = tiny_problem(24, 2, 5, seed=17)
    nf = 6
    delta = orc.transition_energies(qp.e_v, qp.e_c)
    prev = None
    for n_eig in (1, 3, 8, 15, 24):
        out = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, n_eig, nf, keep=True)
        for k in range(nf):
            lam = np.linalg.eigvalsh(orc.chi_tilde(A, qp.qg2, delta, out["omega"][k], qp.omega_cell))
            mu = np.sort(out["lam_k"][k])
            tol = 1e-12 * abs(lam).max()
            assert np.all(mu >= lam[:n_eig] - tol)
            assert np.all(mu <= lam[qp.n_g - n_eig:] + tol)
        if prev is not None:
            assert np.all(out["e_k"] <= prev["e_k"] + 1e-12 * abs(out["e_k"]).max())
            assert out["ec"] <= prev["ec"] + 1e-12 * abs(out["ec"])
        prev = out
    full = orc.ecorr_full_basis(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, nf)
    assert abs(prev["ec"] - full) < 1e-11 * abs(full)


# --- mutation tests: a planted mistake must be caught by the pins -------------

def _run_pins():
    fails = 0
    for fn in (test_chi0_bruteforce_loops, test_rank1_eigenvalue_per_node,
               test_full_basis_equivalence_lu, test_chis_static_is_diagonal_lambda,
               test_projection_bruteforce, test_quadrature_integrates_lorentzian,
               test_subspace_interlacing_bounds_and_monotone_energy,
               lambda: test_quadrature_exact_for_polynomials(8)):
        try:
            fn()
        except AssertionError:
            fails += 1
    return fails


def test_pins_pass_unmutated():
    assert _run_pins() == 0


@pytest.mark.parametrize("mutation", ["transpose_chi0", "drop_antiresonant", "wrong_weight_jacobian",
                                      "project_no_conj", "sign_trace", "chi_s_static_weights"])
def test_planted_mistake_is_caught(monkeypatch, mutation):
    if mutation == "transpose_chi0":
        orig = orc.chi0
        monkeypatch.setattr(orc, "chi0", lambda *a, **k: orig(*a, **k).T)
    elif mutation == "drop_antiresonant":
        monkeypatch.setattr(orc, "freq_weight",
                            lambda d, o, ow=None: 2.0 * np.asarray(d) / (np.asarray(d) ** 2 + o * o))
    elif mutation == "wrong_weight_jacobian":
        orig = orc.frequency_grid
        def fg(n, s=0.5):
            om, wt = orig(n, s)
            return om, wt * (1 + om / (s + om))
        monkeypatch.setattr(orc, "frequency_grid", fg)
    elif mutation == "project_no_conj":
        monkeypatch.setattr(orc, "project",
                            lambda A, qg2, C, vg=None: (np.asarray(A) @ (np.sqrt(orc.coulomb(qg2))[:, None] * C)).T)
    elif mutation == "sign_trace":
        orig = orc.trace_term
        monkeypatch.setattr(orc, "trace_term", lambda *a, **k: -orig(*a, **k))
    elif mutation == "chi_s_static_weights":
        # chi_s(iw_k) built with the omega = 0 weights at every node
        orig = orc.chi_s
        monkeypatch.setattr(orc, "chi_s",
                            lambda Mt, d, o, oc, ow=None: orig(Mt, d, 0.0, oc, ow))
    assert _run_pins() > 0
