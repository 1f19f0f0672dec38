"""GPU checks of the subspace eigensolver's building blocks on their own (step a3):
the Householder tridiagonalisation that starts it (FP32 and FP64) and the Jacobi
solver of its Rayleigh-Ritz step, against LAPACK on seeded Hermitian matrices.

The tridiagonalisation is a unitary similarity, so T has A's eigenvalues; the sizes
span one and several 32-column panels and grids from a few rows per CTA to many, in
both precisions.  The Jacobi solver is checked on full random matrices and on nearly
diagonal ones (its use), including odd sizes, where one player of every round is
paired with the padding index and must still take the other pairs' row rotations.
"""
import numpy as np
import pytest

from paper_2405_20258_gb300 import rpa

pytestmark = pytest.mark.gpu


def hermitian(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return (x + x.conj().T) / 2


@pytest.mark.parametrize("bits", [64, 32])
@pytest.mark.parametrize("n", [1, 2, 33, 64, 100, 300, 1024, 2000])
def test_tridiagonal_keeps_the_spectrum(n, bits):
    import torch
    h = hermitian(n, 11 + n)
    ct, rt = (torch.complex128, torch.float64) if bits == 64 else (torch.complex64, torch.float32)
    # column-major on the device: the rows of the transpose
    a = torch.tensor(np.ascontiguousarray(h.T), dtype=ct, device="cuda")
    d = torch.zeros(n, dtype=rt, device="cuda")
    e = torch.zeros(max(n - 1, 1), dtype=rt, device="cuda")
    rpa.rpa_tridiagonalize(a, d, e)
    torch.cuda.synchronize()
    dd = d.cpu().double().numpy()
    ee = e.cpu().double().numpy()[: n - 1]
    t = np.diag(dd) + np.diag(ee, 1) + np.diag(ee, -1)
    w = np.linalg.eigvalsh(t)
    ref = np.linalg.eigvalsh(h)
    err = np.max(np.abs(w - ref)) / np.max(np.abs(ref))
    tol = 1e-12 if bits == 64 else 2e-5
    print("n=%d bits=%d: eigenvalues of T within %.2e of A's" % (n, bits, err))
    assert err < tol


@pytest.mark.parametrize("m,kind", [(1, "full"), (2, "full"), (7, "full"), (8, "full"),
                                    (9, "full"), (64, "full"), (101, "near"), (500, "near"),
                                    (501, "near")])
def test_jacobi_eigenpairs(m, kind):
    import torch
    h = hermitian(m, 5 + m)
    if kind == "near":
        # like a Rayleigh-Ritz matrix: graded diagonal, small off-diagonal part
        h = np.diag(-np.geomspace(1e3, 1.0, m)) + 1e-3 * h
    g = torch.tensor(np.ascontiguousarray(h.T), dtype=torch.complex128, device="cuda")
    theta = torch.zeros(m, dtype=torch.float64, device="cuda")
    y = torch.zeros((m, m), dtype=torch.complex128, device="cuda")
    rpa.rpa_hermitian_eig_jacobi(g, theta, y)
    torch.cuda.synchronize()
    th = theta.cpu().numpy()
    Y = y.cpu().numpy().T  # column-major on the device
    ref = np.linalg.eigvalsh(h)
    scale = np.max(np.abs(ref))
    err_lam = np.max(np.abs(th - ref)) / scale
    orth = np.max(np.abs(Y.conj().T @ Y - np.eye(m)))
    resid = np.max(np.abs(h @ Y - Y * th[None, :])) / scale
    print("m=%d %s: eigenvalues %.2e, orthonormality %.2e, residual %.2e" %
          (m, kind, err_lam, orth, resid))
    # the rotations' FP64 rounding accumulates in Y as ~m eps (measured 1.0e-13 at m = 501)
    assert err_lam < 1e-13
    assert orth < max(1e-13, 5e-16 * m)
    assert resid < 1e-13
