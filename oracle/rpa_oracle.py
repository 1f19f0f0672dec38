"""FP64 CPU oracle of the static-subspace RPA correlation energy.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  The CUDA path
never calls it and shares no code with it; inputs come from the seeded
generator in ``paper_2405_20258_gb300.inputs`` and are passed in as arrays.

Every function is a plain restatement of one passage of Weinberg et al.,
"Static subspace approximation for random phase approximation correlation
energies" (arXiv:2405.20258), in float64/complex128 with NumPy/LAPACK as the
only primitives (matmul, eigh, slogdet, cholesky).  No blocking, fusion or
reordering beyond what the equations state.

Notation (one q-point):
  A[vc, g] = M_vc(G_g)  plane-wave matrix elements, Eq. (pwMat); row vc = v*N_c + c
  Delta_vc = E_c[c] - E_v[v] > 0
  f_vc(w)  = 4 Delta_vc / (Delta_vc^2 + w^2)   transition weight on the imaginary axis
  v_g      = 4 pi / |q + G_g|^2                 bare Coulomb kernel, Eq. (rpaE)
  chi0(iw) = -(1/Omega) A^H diag(f(w)) A        Eq. (chi0_partial_occs), integer occupations
  chi~     = v^1/2 chi0 v^1/2                   symmetrised so that Tr ln(1 - chi0 v) = ln det(1 - chi~)

Readings of the paper (each listed in the design notes):
  * f_vc: the paper's Delta_vck(q, w) = 2 g_k (f_c - f_v) / (e_c - e_v - iw) keeps
    only the resonant term; adding the anti-resonant partner with f_v = 1,
    f_c = 0, g_k = 1 gives -4 Delta / (Delta^2 + w^2), i.e. chi0 = -(1/Omega) sum f M* M.
  * The subspace is spanned by the N_eig eigenvectors of chi~(0) with the most
    negative eigenvalues (chi~ <= 0, so these are the greatest |lambda|).
  * The trace in Eq. (rpaE) is evaluated from the eigenvalues of the subspace
    matrix chi_s(iw_k) = C^H chi~(iw_k) C, with log1p(-lambda) + lambda per eigenvalue.
  * Frequency quadrature: Gauss-Legendre nodes x on [-1, 1], t = (x + 1)/2,
    w = s t / (1 - t), weight (w_GL / 2) * s / (1 - t)^2, s = 0.5 Ha.

Extensions (next rows of the scope): pair weights w_vck = g_k (f_v - f_c) for
partial occupations and several k-points folded into the transition axis
(Eq. chi0_partial_occs), and an optional slab-truncated Coulomb kernel.

Parity pins (tests/test_oracle_pins.py): Hermitian and negative semidefinite
chi0; closed-form rank-1 energy; full-basis equivalence against an LU
log-determinant of the full matrix; chi_s(0) = diag(lambda); Sylvester
log-determinant identity; polynomial exactness of the quadrature; brute-force
loops on tiny inputs; Cauchy interlacing of chi_s(iw) = C^H chi~(iw) C against
chi~(iw) at every node, with E_c non-increasing in N_eig towards the full-basis
value.  Those bound the truncation error at N_eig < N_G, but its size has no
closed form: parity unpinned beyond this oracle for that quantity.
"""
from __future__ import annotations

import math

import numpy as np

FOUR_PI = 4.0 * math.pi


# --- basic quantities ------------------------------------------------------

def coulomb(qg2):
    """v(G) = 4 pi / |q+G|^2 (bare Coulomb interaction named in Eq. (rpaE))."""
    return FOUR_PI / np.asarray(qg2, dtype=np.float64)


def coulomb_slab(qg_vec, z_c):
    """Slab-truncated Coulomb kernel: the Fourier transform of 1/r cut off at
    |z| > z_c, for (q+G)_z on the reciprocal lattice of a cell of height 2 z_c:
    v = 4 pi/|q+G|^2 [1 - exp(-|q+G|_par z_c) cos((q+G)_z z_c)]  (Ismail-Beigi 2006).
    The paper's surfaces are slabs with vacuum (Computational Details); it names no
    truncation, so this is offered as an option."""
    k = np.asarray(qg_vec, dtype=np.float64)
    kpar = np.hypot(k[:, 0], k[:, 1])
    k2 = np.sum(k * k, axis=1)
    return FOUR_PI / k2 * (1.0 - np.exp(-kpar * z_c) * np.cos(k[:, 2] * z_c))


def transition_energies(e_v, e_c):
    """Delta_vc = e_c - e_v (Eq. (chi0_partial_occs) index pair).  1-D inputs: row
    vc = v * N_c + c; 2-D inputs [n_k][n_v], [n_k][n_c]: k-points folded into the
    transition axis, row (k * N_v + v) * N_c + c."""
    e_v = np.atleast_2d(np.asarray(e_v, dtype=np.float64))
    e_c = np.atleast_2d(np.asarray(e_c, dtype=np.float64))
    return (e_c[:, None, :] - e_v[:, :, None]).reshape(-1)


def pair_weights(occ_v, occ_c, k_weight=None):
    """w_vck = g_k (f_v - f_c): k-point weight times occupation difference of
    Eq. (chi0_partial_occs) (Delta_vck's numerator up to the spin factor), in the
    row order of transition_energies.  Integer occupations (1, 0) give 1."""
    occ_v = np.atleast_2d(np.asarray(occ_v, dtype=np.float64))
    occ_c = np.atleast_2d(np.asarray(occ_c, dtype=np.float64))
    g = np.ones(occ_v.shape[0]) if k_weight is None else np.asarray(k_weight, dtype=np.float64)
    return (g[:, None, None] * (occ_v[:, :, None] - occ_c[:, None, :])).reshape(-1)


def freq_weight(delta, omega, ow=None):
    """f_vc(w) = w_vc 4 Delta / (Delta^2 + w^2): resonant plus anti-resonant term of
    Delta_vck(q, iw) with spin factor 2 (sign carried by chi0); w_vc = g_k (f_v - f_c)
    (1 for integer occupations)."""
    delta = np.asarray(delta, dtype=np.float64)
    f = 4.0 * delta / (delta * delta + omega * omega)
    return f if ow is None else np.asarray(ow, dtype=np.float64) * f


def frequency_grid(n_freq: int, omega_scale: float = 0.5):
    """Gauss-Legendre quadrature on the imaginary axis (n_freq points, Computational Details).

    Returns (omega[n], weight[n]) with  int_0^inf g(w) dw ~= sum_k weight_k g(omega_k).
    """
    x, w = np.polynomial.legendre.leggauss(n_freq)
    t = 0.5 * (x + 1.0)
    omega = omega_scale * t / (1.0 - t)
    weight = 0.5 * w * omega_scale / (1.0 - t) ** 2
    return omega, weight


# --- full-basis polarizability ---------------------------------------------

def chi0(A, delta, omega, omega_cell, ow=None):
    """chi0_GG'(q, iw) = -(1/Omega) sum_vc f_vc(w) conj(M_vc(G)) M_vc(G')  (Eq. chi0_partial_occs)."""
    A = np.asarray(A, dtype=np.complex128)
    f = freq_weight(delta, omega, ow)
    return -(A.conj().T @ (f[:, None] * A)) / omega_cell


def chi_tilde(A, qg2, delta, omega, omega_cell, ow=None, vg=None):
    """chi~ = v^1/2 chi0 v^1/2, Hermitised as (X + X^H)/2 (vg: Coulomb kernel, default bare)."""
    s = np.sqrt(coulomb(qg2) if vg is None else np.asarray(vg, dtype=np.float64))
    x = s[:, None] * chi0(A, delta, omega, omega_cell, ow) * s[None, :]
    return 0.5 * (x + x.conj().T)


# --- subspace ----------------------------------------------------------------

def canonical_gauge(C):
    """Fix each eigenvector's phase: its entry of largest modulus (lowest row on
    ties) is made real and positive."""
    C = np.array(C, dtype=np.complex128, copy=True)
    if C.size == 0:
        return C
    idx = np.argmax(np.abs(C), axis=0)
    ph = C[idx, np.arange(C.shape[1])]
    return C * (np.abs(ph) / ph)[None, :]


def subspace_basis(chit, n_eig):
    """The N_eig eigenvectors of chi~(0) with the greatest |lambda| (most negative,
    since chi~ <= 0), ascending in lambda, in the canonical gauge (Method, C_s)."""
    lam, vec = np.linalg.eigh(chit)
    return lam[:n_eig].copy(), canonical_gauge(vec[:, :n_eig]), lam


def project(A, qg2, C, vg=None):
    """Projected matrix elements M~ = (A v^1/2 C)^H, shape [N_eig, N_vc]  (M_s = M C_s)."""
    B = np.sqrt(coulomb(qg2) if vg is None else np.asarray(vg, dtype=np.float64))[:, None] * C
    return (np.asarray(A, dtype=np.complex128) @ B).conj().T


def chi_s(Mt, delta, omega, omega_cell, ow=None):
    """Subspace polarizability chi_s(iw) = -(1/Omega) M~ diag(f(w)) M~^H  (chi0_s = M_s^+ Delta M_s)."""
    f = freq_weight(delta, omega, ow)
    return -(Mt * f[None, :]) @ Mt.conj().T / omega_cell


def trace_term(Mt, delta, omega, omega_cell, ow=None):
    """Tr chi_s(iw) = -(1/Omega) sum_vc f_vc(w) ||M~[:, vc]||^2 (the chi0 v term of Eq. rpaE)."""
    f = freq_weight(delta, omega, ow)
    return -float(np.sum(f * np.sum(np.abs(Mt) ** 2, axis=0))) / omega_cell


def freq_energy(lam):
    """sum_lambda [ln(1 - lambda) + lambda] for one frequency (Eq. rpaE, trace in the subspace)."""
    lam = np.asarray(lam, dtype=np.float64)
    return float(np.sum(np.log1p(-lam) + lam))


def logdet_cholesky(chis):
    """ln det(1 - chi_s) from a Cholesky factor (1 - chi_s is Hermitian positive
    definite); the determinant route of Implementation, Tr ln = ln det."""
    n = chis.shape[0]
    L = np.linalg.cholesky(np.eye(n) - chis)
    return float(2.0 * np.sum(np.log(np.real(np.diag(L)))))


# --- the whole path ----------------------------------------------------------

def ecorr(A, qg2, e_v, e_c, omega_cell, n_eig, n_freq, omega_scale=0.5, keep=False, ow=None,
          vg=None):
    """Static-subspace RPA correlation energy of one q-point (Method + Implementation).

    Steps in the paper's order: chi0(0) -> chi~(0) -> C_s -> M~ -> chi_s(iw_k)
    for every quadrature node -> eigenvalues -> E_c = (1/2pi) sum_k w_k sum [ln(1-l)+l].
    ow: pair weights g_k (f_v - f_c) (default 1); vg: Coulomb kernel (default bare).
    Returns a dict with E_c and (if ``keep``) every intermediate.
    """
    delta = transition_energies(e_v, e_c)
    chit = chi_tilde(A, qg2, delta, 0.0, omega_cell, ow, vg)
    lam0, C, lam_all = subspace_basis(chit, n_eig)
    Mt = project(A, qg2, C, vg)
    omega, weight = frequency_grid(n_freq, omega_scale)
    lam_k = np.empty((n_freq, n_eig))
    trace_k = np.empty(n_freq)
    e_k = np.empty(n_freq)
    chis_all = [] if keep else None
    for k in range(n_freq):
        chis = chi_s(Mt, delta, omega[k], omega_cell, ow)
        chis = 0.5 * (chis + chis.conj().T)
        lam = np.linalg.eigvalsh(chis)
        lam_k[k] = lam
        trace_k[k] = trace_term(Mt, delta, omega[k], omega_cell, ow)
        e_k[k] = float(np.sum(np.log1p(-lam))) + trace_k[k]
        if keep:
            chis_all.append(chis)
    ec = float(np.sum(weight * e_k)) / (2.0 * math.pi)
    out = dict(ec=ec, e_k=e_k, omega=omega, weight=weight, lam0=lam0, lam_k=lam_k,
               trace_k=trace_k, gap=(float(lam_all[n_eig] - lam_all[n_eig - 1])
                                     if n_eig < len(lam_all) else float("inf")))
    if keep:
        out.update(chit=chit, C=C, Mt=Mt, chis=np.array(chis_all), lam_all=lam_all)
    return out


def ecorr_full_basis(A, qg2, e_v, e_c, omega_cell, n_freq, omega_scale=0.5, ow=None, vg=None):
    """E_c of Eq. (rpaE) in the full G basis, trace of the log by an LU
    log-determinant: Tr ln(1 - chi0 v) = ln det(1 - chi~) (Implementation)."""
    delta = transition_energies(e_v, e_c)
    omega, weight = frequency_grid(n_freq, omega_scale)
    tot = 0.0
    for k in range(n_freq):
        x = chi_tilde(A, qg2, delta, omega[k], omega_cell, ow, vg)
        sign, ld = np.linalg.slogdet(np.eye(x.shape[0]) - x)
        tot += weight[k] * (ld + float(np.real(np.trace(x))))
    return tot / (2.0 * math.pi)
