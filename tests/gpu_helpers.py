"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and return every intermediate on the host, and align eigenvector phases."""
import numpy as np


def run_gpu(qp, A, n_eig, n_freq, precision=0, route="eig", keep=True, generate=False, m_dtype=None,
            slices=(0, 0, 0), **extra):
    """route: "eig" (eigenvalues of every chi_s, returned as lam_k) or "cholesky"."""
    import torch
    from paper_2405_20258_gb300 import rpa

    want_lam = route == "eig"
    route = rpa.RPA_ROUTE_EIG if want_lam else rpa.RPA_ROUTE_CHOLESKY

    dq = rpa.device_qpoint(qp, n_eig, n_freq, A=None if generate else A,
                           m_dtype=m_dtype, **extra)
    n_g, n_vc = qp.n_g, qp.n_vc
    dev = "cuda"
    out = {}
    with rpa.Plan([dq], precision=precision, energy_route=route, slices=slices) as plan:
        chi = torch.empty((n_g, n_g), dtype=torch.complex128, device=dev) if keep else None
        lam0 = torch.empty(n_eig, dtype=torch.float64, device=dev) if keep else None
        C = torch.empty((n_g, n_eig), dtype=torch.complex128, device=dev) if keep else None
        mt = torch.empty((n_eig, n_vc), dtype=torch.complex128, device=dev) if keep else None
        chis = torch.empty((n_freq, n_eig, n_eig), dtype=torch.complex128, device=dev) if keep else None
        tr = torch.empty(n_freq, dtype=torch.float64, device=dev) if keep else None
        lam = torch.empty((n_freq, n_eig), dtype=torch.float64, device=dev) if keep and want_lam else None
        plan.chi0_static(0, chi)
        plan.subspace_basis(0, lam0, C)
        plan.chi_freq(0, mt, chis, tr)
        out["ec"] = plan.ecorr(0, lam)
        out["omega"], out["weight"] = plan.frequencies(0)
        torch.cuda.synchronize()
        for k, v in (("chit", chi), ("lam0", lam0), ("C", C), ("Mt", mt), ("chis", chis),
                     ("trace_k", tr), ("lam_k", lam)):
            if v is not None:
                out[k] = v.cpu().numpy()
    return out


def phases(C_ref, C_gpu):
    """Per-column unit phases ph with C_gpu ~= C_ref * ph."""
    s = np.sum(np.conj(C_ref) * C_gpu, axis=0)
    return s / np.abs(s)


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
