"""The allocation-free trace term, rpa_trace_term_static.

Some callers cannot allocate device memory where they call this library: an
application whose device memory is fully reserved by its own pool allocator,
or code that must not cause the device-wide synchronisation cudaMalloc and
cudaFree can bring.  For them the library offers the trace term of the
subspace polarizability with its scratch in a fixed library array.

This test calls that entry point through the C ABI twice in a row on the same
inputs and checks both results against the trace rpa_chi_freq computes with
its plan-owned workspace, within the 1e-12 relative tolerance of the FP64
parity tests, and against the oracle's trace term on the same M~; then once
more on a smaller problem (the fixed scratch still
holds the larger problem's values), and checks that sizes beyond the fixed
scratch are refused.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2405_20258_gb300 import inputs

pytestmark = pytest.mark.gpu


def plan_trace(n_g, n_v, n_c, n_eig, n_freq):
    import torch
    from paper_2405_20258_gb300 import rpa
    qp = inputs.make_qpoint(n_g, n_v, n_c)
    A = inputs.matrix_elements(qp)
    dq = rpa.device_qpoint(qp, n_eig, n_freq, A=A)
    mt = torch.empty((n_eig, n_v * n_c), dtype=torch.complex128, device="cuda")
    tr = torch.empty(n_freq, dtype=torch.float64, device="cuda")
    with rpa.Plan([dq]) as plan:
        plan.chi0_static(0)
        plan.subspace_basis(0)
        plan.chi_freq(0, mt, None, tr)
        omega, _ = plan.frequencies(0)
    torch.cuda.synchronize()
    return dq, mt, tr.cpu().numpy(), torch.as_tensor(omega, device="cuda")


def static_trace(dq, mt, omega):
    import torch
    from paper_2405_20258_gb300 import rpa
    out = torch.full((omega.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
    rpa.rpa_trace_term_static(mt, mt.shape[0], dq.e_v.shape[0], dq.e_c.shape[0], dq.e_v, dq.e_c,
                              omega, omega.shape[0], dq.omega_cell, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_static_trace_matches_plan_trace():
    from paper_2405_20258_gb300 import rpa
    import oracle.rpa_oracle as orc
    dq, mt, ref, omega = plan_trace(160, 6, 50, 30, 7)
    delta = orc.transition_energies(dq.e_v.cpu().numpy(), dq.e_c.cpu().numpy())
    mt_h, om_h = mt.cpu().numpy(), omega.cpu().numpy()
    ref_orc = np.array([orc.trace_term(mt_h, delta, w, dq.omega_cell) for w in om_h])
    for _ in range(2):
        got = static_trace(dq, mt, omega)
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-12
        assert np.max(np.abs(got - ref_orc) / np.abs(ref_orc)) < 1e-12
    # a smaller problem after the larger one: stale scratch entries are never read
    dq2, mt2, ref2, omega2 = plan_trace(90, 2, 30, 12, 3)
    got2 = static_trace(dq2, mt2, omega2)
    assert np.max(np.abs(got2 - ref2) / np.abs(ref2)) < 1e-12
    # more transitions than the fixed scratch holds: refused before any launch
    import torch
    n_c_big = rpa.STATIC_TRACE_MAX_VC // dq.e_v.shape[0] + 1
    out = torch.zeros(omega.shape[0], dtype=torch.float64, device="cuda")
    with pytest.raises(rpa.RPAError) as e:
        rpa.rpa_trace_term_static(mt, mt.shape[0], dq.e_v.shape[0], n_c_big, dq.e_v, dq.e_c,
                                  omega, omega.shape[0], dq.omega_cell, out)
    assert e.value.status == rpa.RPA_EINVAL
    assert "fixed scratch" in str(e.value)
