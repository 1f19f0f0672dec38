"""The C-ABI library loads on a machine without a GPU, exports every symbol
include/rpa.h declares, and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2405_20258_gb300 import rpa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "rpa.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(rpa_\w+)\(", txt, re.M)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(rpa.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return rpa.load()


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(rpa.EXPORTED)


def test_version_and_status_strings(lib):
    assert b"sm_103a" in lib.rpa_version()
    assert lib.rpa_status_string(rpa.RPA_ESTATE) == b"stage called out of order"


def _q(**kw):
    base = dict(n_g=10, n_v=2, n_c=3, n_eig=4, n_freq=8, omega_cell=1000.0,
                qg2=1, e_v=1, e_c=1, m=1, m_dtype=0, iq=0, seed=0, miller=None)
    base.update(kw)
    return rpa.rpa_qpoint(**base)


@pytest.mark.parametrize("bad,msg", [
    (dict(n_eig=11), "n_eig"), (dict(n_eig=0), "n_eig"), (dict(n_g=0), "n_g"),
    (dict(n_freq=0), "n_freq"), (dict(n_freq=300), "n_freq"), (dict(omega_cell=-1.0), "omega_cell"),
    (dict(qg2=None), "device pointers"), (dict(m_dtype=5), "m_dtype"),
    (dict(m=None), "miller"), (dict(n_v=0), "n_v"), (dict(n_k=-1), "n_k"),
    (dict(coulomb=3), "coulomb"), (dict(coulomb=1, slab_zc=5.0), "qg_vec"),
    (dict(coulomb=1, qg_vec=1, slab_zc=0.0), "slab_zc")])
def test_plan_create_rejects_bad_descriptors(lib, bad, msg):
    q = _q(**bad)
    h = ctypes.c_void_p()
    st = lib.rpa_plan_create(ctypes.byref(h), ctypes.byref(q), 1, None, None)
    assert st == rpa.RPA_EINVAL
    assert h.value is None
    assert msg in lib.rpa_last_error(None).decode()


def test_plan_create_rejects_bad_options(lib):
    q = _q()
    h = ctypes.c_void_p()
    opt = rpa.rpa_options(7, 0, 0.5)
    assert lib.rpa_plan_create(ctypes.byref(h), ctypes.byref(q), 1, ctypes.byref(opt), None) == rpa.RPA_EINVAL
    opt = rpa.rpa_options(0, 9, 0.5)
    assert lib.rpa_plan_create(ctypes.byref(h), ctypes.byref(q), 1, ctypes.byref(opt), None) == rpa.RPA_EINVAL
    assert lib.rpa_plan_create(ctypes.byref(h), ctypes.byref(q), 0, None, None) == rpa.RPA_EINVAL
    assert lib.rpa_plan_create(None, ctypes.byref(q), 1, None, None) == rpa.RPA_EINVAL


def test_null_plan_calls(lib):
    assert lib.rpa_chi0_static(None, 0, None) == rpa.RPA_EINVAL
    assert lib.rpa_ecorr(None, 0, None, None) == rpa.RPA_EINVAL
    assert lib.rpa_plan_destroy(None) == rpa.RPA_EINVAL
    assert lib.rpa_generate_m(None, 0, 1, 0, 1, None, 0, None) == rpa.RPA_EINVAL


def test_building_blocks_reject_bad_arguments(lib):
    # every case fails its argument check before any CUDA call, so no device is needed;
    # the non-NULL pointers below are never dereferenced
    p = ctypes.c_void_p(256)
    assert lib.rpa_tridiagonalize(0, 64, p, p, p, None) == rpa.RPA_EINVAL
    assert lib.rpa_tridiagonalize(8, 16, p, p, p, None) == rpa.RPA_EINVAL
    assert lib.rpa_tridiagonalize(8, 32, None, p, p, None) == rpa.RPA_EINVAL
    assert lib.rpa_tridiagonalize(8, 32, p, p, None, None) == rpa.RPA_EINVAL
    assert lib.rpa_hermitian_eig_jacobi(0, p, p, p, None) == rpa.RPA_EINVAL
    assert lib.rpa_hermitian_eig_jacobi(4, p, None, p, None) == rpa.RPA_EINVAL
    order = lib.rpa_transition_order
    assert order(0, 1, 1, 0, p, p, p, None) == rpa.RPA_EINVAL          # no transitions
    assert order(6, 0, 6, 0, p, p, p, None) == rpa.RPA_EINVAL          # n_v < 1
    assert order(6, 2, 3, 3, p, p, p, None) == rpa.RPA_EINVAL          # seg_bands > n_v
    assert order(6, 2, 3, -1, p, p, p, None) == rpa.RPA_EINVAL         # seg_bands < 0
    assert order(10, 2, 3, 1, p, p, p, None) == rpa.RPA_EINVAL         # not k x n_v x n_c
    assert order(6, 2, 3, 0, None, p, p, None) == rpa.RPA_EINVAL       # NULL delta
    assert order(6, 2, 3, 0, p, p, None, None) == rpa.RPA_EINVAL       # NULL order
    assert b"rpa_transition_order" in lib.rpa_last_error(None)
