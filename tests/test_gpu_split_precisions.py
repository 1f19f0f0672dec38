"""GPU checks of the split precisions (config 3's comparison variants): every
contraction on round-to-nearest hi/lo planes summed in FP32 over K -- BF16 with 3
products (RPA_MIXED_BF16X3) or 6 (RPA_MIXED_BF16X6), TF32 on kind::tf32 tensor
cores with 3 (RPA_MIXED_TF32X3).  They do not reach 1e-6 Ha: at N_G = 4000 the BF16
variants sit ~21 Ha (6e-6 relative) from the FP64 path, the FP32 sums over K
dominating.  Checked here at N_G = 400 against the oracle: each within 2e-5
relative, the exact-digit default within 1e-6 Ha, and the variants distinct from
one another (each ran its own arithmetic)."""
import numpy as np
import pytest

import oracle.rpa_oracle as orc
from paper_2405_20258_gb300 import inputs
from tests.gpu_helpers import run_gpu

pytestmark = pytest.mark.gpu


def test_split_precisions_against_oracle_400():
    from paper_2405_20258_gb300 import rpa
    qp = inputs.make_qpoint(400, 16, 200)
    A = inputs.matrix_elements(qp)
    ref = orc.ecorr(A, qp.qg2, qp.e_v, qp.e_c, qp.omega_cell, 200, 32)["ec"]
    got = {}
    for name in ("RPA_MIXED", "RPA_MIXED_BF16X3", "RPA_MIXED_BF16X6", "RPA_MIXED_TF32X3"):
        ec = run_gpu(qp, A, 200, 32, precision=getattr(rpa, name), keep=False)["ec"]
        got[name] = ec
        print(name, "E_c %.9f  dE_c %.3e Ha (%.2e relative)" % (ec, ec - ref, abs(ec - ref) / abs(ref)))
    assert abs(got["RPA_MIXED"] - ref) <= 1e-6
    for name in ("RPA_MIXED_BF16X3", "RPA_MIXED_BF16X6", "RPA_MIXED_TF32X3"):
        assert np.isfinite(got[name]) and abs(got[name] - ref) <= 2e-5 * abs(ref), name
    assert len({got[k] for k in got}) == 4
