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


def stable_order(delta, ow, n_v, n_c, seg_bands):
    """The permutation the K-blocks of the mixed chi~(0) take: numpy's stable argsort
    of the negated keys, per segment of seg_bands valence bands when seg_bands > 0."""
    key = np.where((ow != 0) & (delta != 0), np.abs(ow / np.where(delta != 0, delta, 1.0)), 0.0)
    if seg_bands == 0:
        return np.argsort(-key, kind="stable")
    out = np.empty(key.size, dtype=np.int64)
    for k in range(key.size // (n_v * n_c)):
        for v0 in range(0, n_v, seg_bands):
            r0 = (k * n_v + v0) * n_c
            rows = min(seg_bands, n_v - v0) * n_c
            out[r0:r0 + rows] = np.argsort(-key[r0:r0 + rows], kind="stable")
    return out


@pytest.mark.parametrize("n_k,n_v,n_c,seg", [(1, 1, 1, 0), (1, 1, 2047, 0), (1, 2, 1024, 0),
                                             (1, 3, 683, 0), (1, 40, 2500, 0), (1, 128, 2000, 0),
                                             (2, 5, 333, 2), (3, 9, 250, 4), (1, 64, 4096, 5)])
def test_transition_order_is_a_stable_sort(n_k, n_v, n_c, seg):
    import torch
    rng = np.random.default_rng(7 + n_v * n_c + seg)
    n = n_k * n_v * n_c
    delta = rng.uniform(0.05, 3.0, n)
    delta[rng.random(n) < 0.1] = 1.0
    ow = rng.choice([0.0, 0.5, 1.0, 2.0], size=n) * np.where(rng.random(n) < 0.5, 1.0,
                                                             rng.uniform(0.9, 1.1, n))
    order = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    rpa.rpa_transition_order(torch.tensor(delta, device="cuda"), torch.tensor(ow, device="cuda"),
                             order, n_v, n_c, seg)
    got = order.cpu().numpy().astype(np.int64)
    assert np.array_equal(got, stable_order(delta, ow, n_v, n_c, seg))
