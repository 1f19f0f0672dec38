"""Seeded synthetic inputs for the static-subspace RPA path.

This module only *draws* inputs: the plane-wave basis of one q-point, the
Kohn-Sham band energies and the plane-wave matrix elements M_vc(G).  It holds
none of the method's arithmetic (no Coulomb kernel, no transition weights, no
polarizability): the same arrays are handed to the CPU oracle and to the CUDA
path, which each do the physics on their own.

Generator (counter-based, so that any sub-block of M can be drawn alone):

* ``splitmix64`` is the published 64-bit mixer of Steele, Lea and Flood
  (OOPSLA 2014, "Fast splittable pseudorandom number generators"): add the
  golden-ratio increment 0x9E3779B97F4A7C15, then two xor-shift-multiply
  rounds (shift 30, multiplier 0xBF58476D1CE4E5B9; shift 27, multiplier
  0x94D049BB133111EB) and a final xor-shift by 31.
* The key of one matrix element is
  ``K = sm(seed ^ sm(sm(((iq << 16) + v) << 32 | c) ^ pack(n1, n2, n3)))``
  with ``pack`` three 21-bit biased Miller indices, so an element is tied to
  its G-vector (not its sorted position) and sub-problems reuse entries.
* Two uniforms ``u_j = ((sm(K ^ 2j) >> 11) + 0.5) * 2**-53`` (j = 0, 1) feed a
  Box-Muller draw ``z = sqrt(-2 ln u0) * exp(2 pi i u1) / sqrt(2)`` (E|z|^2 = 1)
  and ``M_vc(G) = z * exp(-|q+G|^2 / 8)``.
* Band energies: ``E_v = -0.8 u``, ``E_c = 0.04 + 2.96 u`` with
  ``u = ((sm(seed ^ sm((tag << 56) ^ (iq << 32) ^ idx)) >> 11) + 0.5) 2**-53``,
  tag 1 for valence and 2 for conduction bands (Ha).

The basis is the N_G reciprocal-lattice vectors G = (n1, n2, n3) 2pi/a of a
cubic cell with the smallest |q+G|; q = (q1, q2, q3) 2pi/a is given in units of
1/20 of 2pi/a so that 400 |q+G|^2 (a/2pi)^2 is an exact integer sort key; ties
are broken by the Miller indices in lexicographic order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
MUL1 = 0xBF58476D1CE4E5B9
MUL2 = 0x94D049BB133111EB
PACK_BIAS = 1 << 20
DEFAULT_SEED = 20240531


def splitmix64_int(x: int) -> int:
    """splitmix64 of one Python integer (reference form, exact)."""
    z = (x + GOLDEN) & MASK64
    z = ((z ^ (z >> 30)) * MUL1) & MASK64
    z = ((z ^ (z >> 27)) * MUL2) & MASK64
    return z ^ (z >> 31)


def splitmix64(x):
    """Vectorised splitmix64 on a uint64 array (wrap-around arithmetic)."""
    z = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MUL1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MUL2)
    return z ^ (z >> np.uint64(31))


def pack_miller(miller) -> np.ndarray:
    """Three 21-bit biased Miller indices in one uint64 (n1 highest)."""
    m = np.asarray(miller, dtype=np.int64) + PACK_BIAS
    return ((m[:, 0].astype(np.uint64) << np.uint64(42))
            | (m[:, 1].astype(np.uint64) << np.uint64(21))
            | m[:, 2].astype(np.uint64))


def unit_uniform(bits) -> np.ndarray:
    """Top 53 bits of a uint64 mapped to the open interval (0, 1)."""
    return ((np.asarray(bits, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53


@dataclass
class QPoint:
    """One q-point of a synthetic workload (all arrays host numpy)."""
    miller: np.ndarray          # int32 [n_g, 3]
    qg2: np.ndarray             # float64 [n_g]  |q+G|^2, bohr^-2
    e_v: np.ndarray             # float64 [n_v]  Ha
    e_c: np.ndarray             # float64 [n_c]  Ha
    iq: int = 0
    seed: int = DEFAULT_SEED
    q_twentieths: tuple = (1, 0, 0)
    a: float = 10.0
    n_k: int = 1                 # k-points folded into the transition axis
    meta: dict = field(default_factory=dict)

    @property
    def n_g(self):
        return int(self.qg2.shape[0])

    @property
    def n_v(self):
        return int(self.e_v.shape[-1])

    @property
    def n_c(self):
        return int(self.e_c.shape[-1])

    @property
    def n_vc(self):
        return self.n_k * self.n_v * self.n_c

    @property
    def omega_cell(self):
        return self.a ** 3


def gvectors(n_g: int, q_twentieths=(1, 0, 0), a: float = 10.0):
    """The n_g Miller indices with the smallest |q+G| and their |q+G|^2.

    ``q_twentieths`` is q in units of (2pi/a)/20, so the default (1, 0, 0)
    is q = (0.05, 0, 0) 2pi/a.  Returns (miller int32 [n_g,3], qg2 f64 [n_g]).
    """
    if n_g <= 0:
        return np.zeros((0, 3), np.int32), np.zeros(0)
    qi = np.asarray(q_twentieths, dtype=np.int64)
    r = int(math.ceil((3.0 * n_g / (4.0 * math.pi)) ** (1.0 / 3.0))) + 3
    while True:
        rng = np.arange(-r, r + 1, dtype=np.int64)
        n1, n2, n3 = np.meshgrid(rng, rng, rng, indexing="ij")
        n = np.stack([n1.ravel(), n2.ravel(), n3.ravel()], axis=1)
        key = ((20 * n + qi) ** 2).sum(axis=1)
        order = np.lexsort((n[:, 2], n[:, 1], n[:, 0], key))
        sel = order[:n_g]
        # the selection is complete if no vector outside the cube could beat it
        kmax = key[sel[-1]]
        inner = (20 * r - np.abs(qi).max()) ** 2
        if kmax < inner:
            break
        r += 4
    miller = n[sel].astype(np.int32)
    qg2 = key[sel].astype(np.float64) / 400.0 * (2.0 * math.pi / a) ** 2
    return miller, qg2


def band_energies(seed: int, n_v: int, n_c: int, iq: int = 0):
    """Valence energies uniform in [-0.8, 0] Ha, conduction in [0.04, 3.0] Ha."""
    def u(tag, n):
        idx = np.arange(n, dtype=np.uint64)
        x = (np.uint64(tag) << np.uint64(56)) ^ (np.uint64(iq) << np.uint64(32)) ^ idx
        return unit_uniform(splitmix64(np.uint64(seed) ^ splitmix64(x)))
    return -0.8 * u(1, n_v), 0.04 + 2.96 * u(2, n_c)


def element_keys(seed: int, iq: int, v, c, packed_g) -> np.ndarray:
    """Counter keys K[v, c, g] (uint64) of the matrix elements."""
    v = np.asarray(v, dtype=np.uint64)[:, None, None]
    c = np.asarray(c, dtype=np.uint64)[None, :, None]
    pg = np.asarray(packed_g, dtype=np.uint64)[None, None, :]
    vc = ((np.uint64(iq) << np.uint64(16)) + v) << np.uint64(32) | c
    return splitmix64(np.uint64(seed) ^ splitmix64(splitmix64(vc) ^ pg))


def matrix_elements(qp: QPoint, v_range=None, c_range=None, dtype=np.complex128) -> np.ndarray:
    """A[vc, g] = M_vc(G_g) for v in v_range, c in c_range (row vc = v*n_c' + c).

    Returns an array of shape [len(v_range)*len(c_range), n_g], G contiguous.
    With n_k > 1 k-points (and no ranges) the rows are [k][v][c]; the bands of
    k-point k carry the generator indices k*n_v + v and k*n_c + c.
    """
    if qp.n_k > 1 and v_range is None and c_range is None:
        return np.concatenate([
            matrix_elements(qp, np.arange(k * qp.n_v, (k + 1) * qp.n_v),
                            np.arange(k * qp.n_c, (k + 1) * qp.n_c), dtype)
            for k in range(qp.n_k)])
    vr = np.arange(qp.n_v) if v_range is None else np.asarray(v_range)
    cr = np.arange(qp.n_c) if c_range is None else np.asarray(c_range)
    pg = pack_miller(qp.miller)
    out = np.empty((len(vr), len(cr), qp.n_g), dtype=dtype)
    env = np.exp(-qp.qg2 / 8.0)
    # draw in slabs of valence bands to bound the temporaries
    step = max(1, int(4_000_000 // max(1, len(cr) * qp.n_g)))
    for s in range(0, len(vr), step):
        k = element_keys(qp.seed, qp.iq, vr[s:s + step], cr, pg)
        u0 = unit_uniform(splitmix64(k))
        u1 = unit_uniform(splitmix64(k ^ np.uint64(2)))
        rad = np.sqrt(-2.0 * np.log(u0)) / math.sqrt(2.0)
        ang = 2.0 * math.pi * u1
        out[s:s + step] = ((rad * np.cos(ang) + 1j * (rad * np.sin(ang))) * env).astype(dtype)
    return out.reshape(len(vr) * len(cr), qp.n_g)


def make_qpoint(n_g: int, n_v: int, n_c: int, seed: int = DEFAULT_SEED, iq: int = 0,
                q_twentieths=(1, 0, 0), a: float = 10.0, n_k: int = 1) -> QPoint:
    """One synthetic q-point; with n_k > 1 the band energies are [n_k][n_v], [n_k][n_c]."""
    miller, qg2 = gvectors(n_g, q_twentieths, a)
    e_v, e_c = band_energies(seed, n_k * n_v, n_k * n_c, iq)
    if n_k > 1:
        e_v, e_c = e_v.reshape(n_k, n_v), e_c.reshape(n_k, n_c)
    return QPoint(miller=miller, qg2=qg2, e_v=e_v, e_c=e_c, iq=iq, seed=seed,
                  q_twentieths=tuple(int(x) for x in q_twentieths), a=a, n_k=n_k)


def fermi_occupations(e, mu: float, sigma: float) -> np.ndarray:
    """Fermi-Dirac occupations 1/(1 + exp((e - mu)/sigma)) of band energies (Ha):
    the smeared occupations a DFT run hands to the RPA step."""
    return 1.0 / (1.0 + np.exp((np.asarray(e, dtype=np.float64) - mu) / sigma))


def qg_vectors(qp: QPoint) -> np.ndarray:
    """Cartesian q+G (bohr^-1) of the q-point's plane waves, [n_g][3]."""
    q = np.asarray(qp.q_twentieths, dtype=np.float64) / 20.0
    return (q[None, :] + qp.miller.astype(np.float64)) * (2.0 * math.pi / qp.a)


def qgrid_4x4x4():
    """q = ((i, j, k)/4 + (0.05, 0, 0)) 2pi/a for i, j, k in 0..3, in 1/20 units."""
    return [(5 * i + 1, 5 * j, 5 * k) for i in range(4) for j in range(4) for k in range(4)]


def batched_workload(n_q: int = 64, seed: int = DEFAULT_SEED, n_v: int = 96,
                     ng_range=(1500, 6000), nc_range=(800, 2400)):
    """Sizes of the uneven multi-q workload: N_G and N_c drawn per q from the
    same counter generator (tags 3 and 4)."""
    qs = qgrid_4x4x4()[:n_q]
    out = []
    for iq, qt in enumerate(qs):
        ug = unit_uniform(splitmix64(np.uint64(seed) ^ splitmix64(np.uint64((3 << 56) | iq))))
        uc = unit_uniform(splitmix64(np.uint64(seed) ^ splitmix64(np.uint64((4 << 56) | iq))))
        n_g = int(ng_range[0] + math.floor(float(ug) * (ng_range[1] - ng_range[0] + 1)))
        n_c = int(nc_range[0] + math.floor(float(uc) * (nc_range[1] - nc_range[0] + 1)))
        out.append(dict(iq=iq, q_twentieths=qt, n_g=n_g, n_v=n_v, n_c=n_c))
    return out
