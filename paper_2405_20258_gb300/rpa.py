"""Thin ctypes binding of ``librpa.so`` (the C ABI declared in include/rpa.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  PyTorch supplies device memory and the stream.  If the library is
missing this module raises on first use; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librpa.so")

RPA_OK, RPA_EINVAL, RPA_ENOMEM, RPA_ECUDA, RPA_EEIG, RPA_ENUMERIC, RPA_ETIMEOUT, RPA_ESTATE = range(8)
RPA_FP64, RPA_MIXED, RPA_MIXED_BF16X3, RPA_MIXED_BF16X6, RPA_MIXED_TF32X3 = 0, 1, 2, 3, 4
RPA_ROUTE_CHOLESKY, RPA_ROUTE_EIG = 0, 1
RPA_C128, RPA_C64 = 0, 1
RPA_COULOMB_BARE, RPA_COULOMB_SLAB = 0, 1

EXPORTED = ("rpa_plan_create", "rpa_plan_destroy", "rpa_last_error", "rpa_status_string",
            "rpa_chi0_static", "rpa_subspace_basis", "rpa_chi_freq", "rpa_ecorr",
            "rpa_plan_frequencies", "rpa_generate_m", "rpa_version", "rpa_plan_timings",
            "rpa_trace_term_static", "rpa_tridiagonalize", "rpa_hermitian_eig_jacobi",
            "rpa_transition_order")
STATIC_TRACE_MAX_VC = 524288
TIMERS = ("chi0", "eig0", "proj", "chis", "trace", "eigs", "energy", "other", "slice")


class rpa_qpoint(ctypes.Structure):
    _fields_ = [("n_g", ctypes.c_int), ("n_v", ctypes.c_int), ("n_c", ctypes.c_int),
                ("n_eig", ctypes.c_int), ("n_freq", ctypes.c_int),
                ("omega_cell", ctypes.c_double),
                ("qg2", ctypes.c_void_p), ("e_v", ctypes.c_void_p), ("e_c", ctypes.c_void_p),
                ("m", ctypes.c_void_p), ("m_dtype", ctypes.c_int), ("iq", ctypes.c_int),
                ("seed", ctypes.c_ulonglong), ("miller", ctypes.c_void_p),
                ("n_k", ctypes.c_int), ("k_weight", ctypes.c_void_p), ("occ_v", ctypes.c_void_p),
                ("occ_c", ctypes.c_void_p), ("coulomb", ctypes.c_int),
                ("slab_zc", ctypes.c_double), ("qg_vec", ctypes.c_void_p)]


class rpa_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("energy_route", ctypes.c_int),
                ("omega_scale", ctypes.c_double), ("timing", ctypes.c_int),
                ("slices_chi0", ctypes.c_int), ("slices_proj", ctypes.c_int),
                ("slices_chis", ctypes.c_int), ("debug_stall", ctypes.c_int),
                ("vc_chunk", ctypes.c_int), ("reserved", ctypes.c_int * 2)]


class RPAError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


_STATUS = {0: "RPA_OK", 1: "RPA_EINVAL", 2: "RPA_ENOMEM", 3: "RPA_ECUDA", 4: "RPA_EEIG",
           5: "RPA_ENUMERIC", 6: "RPA_ETIMEOUT", 7: "RPA_ESTATE"}
_lib = None


def load(path: str = LIB_PATH):
    """Load librpa.so once; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("librpa.so not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "rpa_plan_create": ([ctypes.POINTER(vp), ctypes.POINTER(rpa_qpoint), i,
                             ctypes.POINTER(rpa_options), vp], i),
        "rpa_plan_destroy": ([vp], i),
        "rpa_last_error": ([vp], ctypes.c_char_p),
        "rpa_status_string": ([i], ctypes.c_char_p),
        "rpa_chi0_static": ([vp, i, vp], i),
        "rpa_subspace_basis": ([vp, i, vp, vp], i),
        "rpa_chi_freq": ([vp, i, vp, vp, vp], i),
        "rpa_ecorr": ([vp, i, vp, vp], i),
        "rpa_plan_frequencies": ([vp, i, vp, vp], i),
        "rpa_generate_m": ([ctypes.POINTER(rpa_qpoint), i, i, i, i, vp, i, vp], i),
        "rpa_version": ([], ctypes.c_char_p),
        "rpa_plan_timings": ([vp, vp, vp], i),
        "rpa_trace_term_static": ([vp, i, i, i, vp, vp, vp, i, d, vp, vp], i),
        "rpa_tridiagonalize": ([i, i, vp, vp, vp, vp], i),
        "rpa_hermitian_eig_jacobi": ([i, vp, vp, vp, vp], i),
        "rpa_transition_order": ([i, i, i, i, vp, vp, vp, vp], i),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _check(status, plan=None):
    if status != RPA_OK:
        msg = load().rpa_last_error(plan).decode()
        raise RPAError(status, msg)


@dataclass
class DeviceQPoint:
    """Device arrays of one q-point (torch tensors kept alive by the plan)."""
    qg2: object
    e_v: object
    e_c: object
    m: object            # complex128/complex64 [n_v*n_c, n_g] or None
    n_eig: int
    n_freq: int
    omega_cell: float = 1000.0
    miller: object = None
    seed: int = 0
    iq: int = 0
    m_dtype: int = RPA_C128
    n_k: int = 1
    k_weight: object = None   # [n_k] float64 or None
    occ_v: object = None      # [n_k, n_v] float64 or None (1)
    occ_c: object = None      # [n_k, n_c] float64 or None (0)
    coulomb: int = RPA_COULOMB_BARE
    slab_zc: float = 0.0
    qg_vec: object = None     # [n_g, 3] float64 (slab kernel)

    def struct(self):
        import torch
        n_g, n_v, n_c = self.qg2.shape[0], self.e_v.shape[-1], self.e_c.shape[-1]
        dt = self.m_dtype
        if self.m is not None:
            dt = RPA_C64 if self.m.dtype == torch.complex64 else RPA_C128
        return rpa_qpoint(n_g, n_v, n_c, self.n_eig, self.n_freq, float(self.omega_cell),
                          _ptr(self.qg2), _ptr(self.e_v), _ptr(self.e_c), _ptr(self.m), dt,
                          int(self.iq), int(self.seed), _ptr(self.miller), int(self.n_k),
                          _ptr(self.k_weight), _ptr(self.occ_v), _ptr(self.occ_c),
                          int(self.coulomb), float(self.slab_zc), _ptr(self.qg_vec))


def device_qpoint(qp, n_eig, n_freq, A=None, device="cuda", m_dtype=None, generate=False,
                  k_weight=None, occ_v=None, occ_c=None, slab_zc=None, qg_vec=None):
    """Upload a host ``inputs.QPoint`` (and optionally A, k-point weights,
    occupations, a slab Coulomb kernel's q+G vectors) to the device."""
    import torch
    f64 = lambda x: None if x is None else torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64),
                                                            device=device)
    dq = DeviceQPoint(
        qg2=torch.as_tensor(qp.qg2, dtype=torch.float64, device=device),
        e_v=torch.as_tensor(qp.e_v, dtype=torch.float64, device=device),
        e_c=torch.as_tensor(qp.e_c, dtype=torch.float64, device=device),
        m=None if A is None else torch.as_tensor(A, device=device),
        n_eig=n_eig, n_freq=n_freq, omega_cell=qp.omega_cell,
        miller=torch.as_tensor(np.ascontiguousarray(qp.miller, dtype=np.int32), device=device),
        seed=qp.seed, iq=qp.iq, n_k=getattr(qp, "n_k", 1),
        k_weight=f64(k_weight), occ_v=f64(occ_v), occ_c=f64(occ_c))
    if slab_zc is not None:
        dq.coulomb, dq.slab_zc, dq.qg_vec = RPA_COULOMB_SLAB, float(slab_zc), f64(qg_vec)
    if m_dtype is not None:
        dq.m_dtype = m_dtype
    return dq


class Plan:
    """Owner of an ``rpa_plan_t``; methods mirror the C entry points."""

    def __init__(self, qpoints, precision=RPA_FP64, energy_route=RPA_ROUTE_CHOLESKY, omega_scale=0.5,
                 stream=None, timing=False, slices=(0, 0, 0), debug_stall=0, vc_chunk=0):
        lib = load()
        self.qpoints = list(qpoints)
        self._structs = (rpa_qpoint * len(self.qpoints))(*[q.struct() for q in self.qpoints])
        opt = rpa_options(precision, energy_route, omega_scale, int(bool(timing)), *slices,
                          int(debug_stall), int(vc_chunk))
        self._stream = _stream(stream)
        h = ctypes.c_void_p()
        st = lib.rpa_plan_create(ctypes.byref(h), self._structs, len(self.qpoints), ctypes.byref(opt),
                                 self._stream)
        if st != RPA_OK:
            raise RPAError(st, lib.rpa_last_error(None).decode())
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            load().rpa_plan_destroy(self.handle)
            self.handle = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def chi0_static(self, iq, chi_out=None):
        _check(load().rpa_chi0_static(self.handle, iq, _ptr(chi_out)), self.handle)

    def subspace_basis(self, iq, lam_out=None, c_out=None):
        _check(load().rpa_subspace_basis(self.handle, iq, _ptr(lam_out), _ptr(c_out)), self.handle)

    def chi_freq(self, iq, mt_out=None, chis_out=None, trace_out=None):
        _check(load().rpa_chi_freq(self.handle, iq, _ptr(mt_out), _ptr(chis_out), _ptr(trace_out)),
               self.handle)

    def ecorr(self, iq, lam_out=None):
        n = len(self.qpoints) if iq == -1 else 1
        out = (ctypes.c_double * n)()
        _check(load().rpa_ecorr(self.handle, iq, ctypes.cast(out, ctypes.c_void_p), _ptr(lam_out)),
               self.handle)
        return list(out) if iq == -1 else out[0]

    def frequencies(self, iq):
        n = self.qpoints[iq].n_freq
        om = np.zeros(n)
        wt = np.zeros(n)
        _check(load().rpa_plan_frequencies(self.handle, iq, om.ctypes.data_as(ctypes.c_void_p),
                                           wt.ctypes.data_as(ctypes.c_void_p)), self.handle)
        return om, wt

    def timings(self):
        """({stage: ms} since the previous call, kernel launches since the previous call)."""
        t = (ctypes.c_double * len(TIMERS))()
        n = ctypes.c_longlong()
        _check(load().rpa_plan_timings(self.handle, ctypes.cast(t, ctypes.c_void_p),
                                       ctypes.cast(ctypes.byref(n), ctypes.c_void_p)), self.handle)
        return dict(zip(TIMERS, list(t))), n.value

    def run(self, iq=0):
        """All stages of one q-point; returns E_c (Ha)."""
        self.chi0_static(iq)
        self.subspace_basis(iq)
        self.chi_freq(iq)
        return self.ecorr(iq)


# names of the C ABI, for callers that prefer the flat form
def rpa_plan_create(qpoints, precision=RPA_FP64, energy_route=RPA_ROUTE_CHOLESKY, omega_scale=0.5,
                    stream=None, timing=False, slices=(0, 0, 0)):
    return Plan(qpoints, precision, energy_route, omega_scale, stream, timing, slices)


def rpa_chi0_static(plan, iq, chi_out=None):
    plan.chi0_static(iq, chi_out)


def rpa_subspace_basis(plan, iq, lam_out=None, c_out=None):
    plan.subspace_basis(iq, lam_out, c_out)


def rpa_chi_freq(plan, iq, mt_out=None, chis_out=None, trace_out=None):
    plan.chi_freq(iq, mt_out, chis_out, trace_out)


def rpa_ecorr(plan, iq, lam_out=None):
    return plan.ecorr(iq, lam_out)


def rpa_plan_destroy(plan):
    plan.close()


def rpa_generate_m(dq: DeviceQPoint, v0, nv, c0, nc, out, stream=None):
    """Draw A[v0:v0+nv, c0:c0+nc, :] on the device into ``out`` (complex128 or complex64)."""
    import torch
    dt = RPA_C64 if out.dtype == torch.complex64 else RPA_C128
    s = dq.struct()
    _check(load().rpa_generate_m(ctypes.byref(s), v0, nv, c0, nc, _ptr(out), dt, _stream(stream)))


def rpa_trace_term_static(mtilde, n_eig, n_v, n_c, e_v, e_c, omega, n_freq, omega_cell, trace_out,
                          stream=None):
    """Trace term of the subspace polarizability without a plan and without any
    device allocation (for callers that cannot allocate): scratch is a fixed
    library array of STATIC_TRACE_MAX_VC doubles.  All arrays are device tensors."""
    _check(load().rpa_trace_term_static(_ptr(mtilde), int(n_eig), int(n_v), int(n_c), _ptr(e_v),
                                        _ptr(e_c), _ptr(omega), int(n_freq), float(omega_cell),
                                        _ptr(trace_out), _stream(stream)))


def rpa_tridiagonalize(a, d, e, stream=None):
    """Householder tridiagonalisation T = Q^H A Q of the square Hermitian device tensor
    a (complex64: FP32, complex128: FP64; read column-major, overwritten with the
    reflectors) into the real device tensors d (n) and e (n - 1)."""
    import torch
    bits = 64 if a.dtype == torch.complex128 else 32
    _check(load().rpa_tridiagonalize(int(a.shape[0]), bits, _ptr(a), _ptr(d), _ptr(e),
                                     _stream(stream)))


def rpa_hermitian_eig_jacobi(g, theta, y, stream=None):
    """All eigenpairs of the Hermitian complex128 device tensor g (m x m, read
    column-major, destroyed) by the library's Jacobi solver: theta (m, ascending) and
    the column-major eigenvectors y (m x m complex128)."""
    _check(load().rpa_hermitian_eig_jacobi(int(g.shape[0]), _ptr(g), _ptr(theta), _ptr(y),
                                           _stream(stream)))


def rpa_transition_order(delta, ow, order, n_v, n_c, seg_bands=0, stream=None):
    """Transition order of the mixed path's chi~(0) K-blocks into the int32 device
    tensor order: the transitions by decreasing |ow / delta| (0 where either is 0),
    equal keys by index; seg_bands > 0 sorts within segments of that many valence
    bands of one k-point, as segment-local indices.  delta, ow: float64 device."""
    _check(load().rpa_transition_order(int(delta.numel()), int(n_v), int(n_c), int(seg_bands),
                                       _ptr(delta), _ptr(ow), _ptr(order), _stream(stream)))


def rpa_version():
    return load().rpa_version().decode()
