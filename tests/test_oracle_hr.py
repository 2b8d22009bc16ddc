"""Pins for the oracle's local H per lattice vector, H_IJ(R) (paper Sec. 2: H(R) and its Bloch
sum H(k) = sum_R e^{ik.R} H(R); Sec. 3.3.1: the local-potential matrix element between phi_mu at
tau_I and phi_nu at tau_J + R).  Checked against the folded Gamma-point oracle (a different code
path: images summed inside the orbitals), the transpose identity, and closed-form two-centre
Gaussian overlaps of single image pairs.
"""
import itertools
import math

import numpy as np

from oracle.oracle import Oracle
from paper_2603_21835_gb300 import inputs
from tests.test_oracle_pins import _SOLID, _gauss_radial, _overlap_1d, _species, _system


def _lattice_vectors(system, I, J, reach):
    """All integer n with |tau_J + n A - tau_I| < reach (the R that can carry an overlap)."""
    A = np.asarray(system.cell, float)
    d = np.asarray(system.pos[J], float) - np.asarray(system.pos[I], float)
    m = int(math.ceil(reach / np.linalg.norm(A, axis=1).min())) + 1
    out = [n for n in itertools.product(range(-m, m + 1), repeat=3) if np.linalg.norm(d + np.array(n) @ A) < reach]
    return np.array(out, dtype=np.int32)


def test_lattice_sum_of_HR_is_the_folded_block():
    """8-atom Si cell (10.26 Bohr, rc 7): images fold, so each block spreads over many R, and
    sum_R H_IJ(R) must equal the folded (Gamma-point) block."""
    w = inputs.config_workload("si8_g48")
    o = Oracle(w.system)
    for I, J in [(0, 0), (0, 5), (3, 7), (6, 2)]:
        R = _lattice_vectors(w.system, I, J, 2 * 7.0 + 0.5)
        HR, missed = o.vlocal_block_R(w.V, I, J, R)
        assert missed == 0.0
        assert len(R) > 1  # several image pairs per block in this cell
        Hf = o.vlocal_block(w.V, I, J)
        assert np.abs(HR.sum(0) - Hf).max() <= 1e-13 * np.abs(Hf).max()
        assert np.abs(HR).max() > 1e-3 * np.abs(Hf).max()


def test_transposed_block_at_minus_R():
    """H_JI(-R) = H_IJ(R)^T."""
    w = inputs.config_workload("si8_g48")
    o = Oracle(w.system)
    I, J = 1, 4
    R = _lattice_vectors(w.system, I, J, 2 * 7.0 + 0.5)
    HIJ, _ = o.vlocal_block_R(w.V, I, J, R)
    HJI, _ = o.vlocal_block_R(w.V, J, I, -R)
    assert np.abs(HJI - HIJ.transpose(0, 2, 1)).max() <= 1e-14 * np.abs(HIJ).max()


def test_incomplete_list_reports_the_missed_products():
    w = inputs.config_workload("si8_g48")
    o = Oracle(w.system)
    R = _lattice_vectors(w.system, 0, 5, 2 * 7.0 + 0.5)
    _, missed = o.vlocal_block_R(w.V, 0, 5, R[:-3])
    assert missed > 0.0


def _closed_form_overlap_R(system, I, J, n):
    """int phi_mu(r - tau_I) phi_nu(r - tau_J - n A) dr for r^l e^{-alpha r^2} Y_lm (one image pair)."""
    def orbs(a, centre):
        out = []
        for rad in system.sp[system.species[a]].radials:
            for poly in _SOLID[rad.l]:
                out.append((centre, rad.alpha, poly))
        return out
    A0 = np.asarray(system.pos[I], float)
    B0 = np.asarray(system.pos[J], float) + np.asarray(n, float) @ np.asarray(system.cell, float)
    oi, oj = orbs(I, A0), orbs(J, B0)
    S = np.zeros((len(oi), len(oj)))
    for i, (A, a, pa) in enumerate(oi):
        for j, (B, b, pb) in enumerate(oj):
            acc = 0.0
            for ea, ca in pa.items():
                for eb, cb in pb.items():
                    acc += ca * cb * np.prod([_overlap_1d(ea[c], eb[c], a, b, A[c], B[c]) for c in range(3)])
            S[i, j] = acc
    return S


def test_HR_with_unit_potential_is_the_closed_form_image_pair_overlap():
    """V = 1 and Gaussian radials r^l e^{-alpha r^2} (support where the tail is below 1e-17): each
    H_IJ(R) is the two-centre overlap of ONE image pair, a closed form (Gaussian product theorem),
    in a 7 Bohr cell where the 7.5 Bohr supports fold many images onto each point."""
    rc = 7.5
    sp = _species([_gauss_radial(0, 0.8, rc), _gauss_radial(1, 1.0, rc), _gauss_radial(2, 1.2, rc)])
    sysm = _system(np.eye(3) * 7.0, [[0.3, 1.1, 0.7], [3.9, 2.2, 4.4]], [0, 0], [sp], (24, 24, 24))
    o = Oracle(sysm, analytic=True)
    V = np.ones(o.ngrid)
    for I, J in [(0, 1), (1, 1)]:
        R = _lattice_vectors(sysm, I, J, 2 * rc)
        HR, missed = o.vlocal_block_R(V, I, J, R)
        assert missed == 0.0
        S = np.stack([_closed_form_overlap_R(sysm, I, J, n) for n in R])
        assert np.abs(HR - S).max() <= 1e-12 * np.abs(S).max()
