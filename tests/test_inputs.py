"""The seeded synthetic-input generator shared by the oracle tests and the CUDA path."""
import math
import os

import numpy as np

from paper_2405_20258_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vectors():
    with open(os.path.join(GOLDEN, "splitmix64_vectors.txt")) as f:
        rows = [list(map(int, l.split())) for l in f if l.strip() and not l.startswith("#")]
    for row in rows:
        state, outs = row[0], row[1:]
        for expect in outs:
            assert inputs.splitmix64_int(state) == expect
            # the vectorised form agrees with the exact integer form
            assert int(inputs.splitmix64(np.array([state], np.uint64))[0]) == expect
            state = (state + inputs.GOLDEN) & inputs.MASK64


def test_gvectors_smallest_and_tiebreak():
    n = 137
    miller, qg2 = inputs.gvectors(n)
    assert miller.shape == (n, 3) and len(np.unique(miller, axis=0)) == n
    key = ((20 * miller.astype(np.int64) + np.array([1, 0, 0])) ** 2).sum(1)
    assert np.all(np.diff(key) >= 0)
    for i in range(n - 1):
        if key[i] == key[i + 1]:
            assert tuple(miller[i]) < tuple(miller[i + 1])
    # brute force: every lattice vector with a smaller key is in the set
    r = 8
    g = np.array([(a, b, c) for a in range(-r, r + 1) for b in range(-r, r + 1) for c in range(-r, r + 1)])
    kall = ((20 * g + np.array([1, 0, 0])) ** 2).sum(1)
    assert np.sum(kall < key[-1]) <= n and np.sum(kall <= key[-1]) >= n
    assert np.allclose(qg2, key / 400.0 * (2 * math.pi / 10.0) ** 2, rtol=0, atol=1e-15)
    assert tuple(miller[0]) == (0, 0, 0)


def test_band_energy_ranges():
    e_v, e_c = inputs.band_energies(inputs.DEFAULT_SEED, 200, 300)
    assert e_v.min() >= -0.8 and e_v.max() <= 0
    assert e_c.min() >= 0.04 and e_c.max() <= 3.0
    assert abs(e_v.mean() + 0.4) < 0.1 and abs(e_c.mean() - 1.52) < 0.3


def test_matrix_elements_statistics_and_subblocks():
    qp = inputs.make_qpoint(50, 8, 40)
    A = inputs.matrix_elements(qp)
    z = A / np.exp(-qp.qg2 / 8.0)[None, :]
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 0.05
    assert abs(np.mean(z.real)) < 0.05 and abs(np.mean(z.imag)) < 0.05
    sub = inputs.matrix_elements(qp, v_range=[3, 5], c_range=[7, 8, 39])
    full = A.reshape(8, 40, 50)
    assert np.array_equal(sub.reshape(2, 3, 50), full[[3, 5]][:, [7, 8, 39]])
    # entries are tied to the G-vector: the first G vectors of a bigger basis draw the same values
    qp2 = inputs.make_qpoint(80, 8, 40)
    A2 = inputs.matrix_elements(qp2)
    assert np.array_equal(A2[:, :50], A)


def test_batched_workload_ranges():
    w = inputs.batched_workload()
    assert len(w) == 64
    assert all(1500 <= x["n_g"] <= 6000 and 800 <= x["n_c"] <= 2400 for x in w)
    assert len({x["q_twentieths"] for x in w}) == 64


def test_qg_vectors_match_qg2_and_grid_offsets():
    qp = inputs.make_qpoint(120, 2, 5, q_twentieths=(6, 5, 0))
    v = inputs.qg_vectors(qp)
    assert np.allclose(np.sum(v ** 2, axis=1), qp.qg2, rtol=1e-14, atol=0)
    grid = inputs.qgrid_4x4x4()
    assert len(grid) == 64 and len(set(grid)) == 64
    # every q of the grid keeps q + G away from zero (the 0.05 offset along x)
    assert all(t[0] % 5 == 1 for t in grid)


def test_fermi_occupations_bounds_and_monotone():
    e = np.linspace(-1.0, 1.0, 101)
    f = inputs.fermi_occupations(e, 0.0, 0.05)
    assert np.all((f >= 0) & (f <= 1)) and np.all(np.diff(f) <= 0)
    assert abs(f[50] - 0.5) < 1e-15 and f[0] > 1 - 1e-8 and f[-1] < 1e-8
