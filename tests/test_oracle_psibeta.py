"""Pins for the oracle's velocity-gauge projector overlaps, P_{j mu}^{IJ}(A) = <beta_{I j}| e^{-i A.r}
|Phi_{J mu}> on an atom-centred spherical grid (paper Sec. 3.3.2, "Spherical Grid Integration for
Nonlocal Potentials").  The paper's 110-point Lebedev-Laikov rule is not available here; its stand-in
is a product rule of the same degree (17): Gauss-Legendre in cos(theta) x uniform azimuth.  Checked
against closed forms (Gaussian product theorem, with and without the plane-wave phase), the exact
moments of the angular rule, translation covariance and the A -> -A conjugation."""
import math

import numpy as np

from oracle.oracle import Oracle
from paper_2603_21835_gb300 import inputs
from tests.test_oracle_pins import _SOLID, _gauss_radial, _overlap_1d, _species, _system


def angular_rule(nt: int = 9, nph: int = 18) -> np.ndarray:
    """[nt * nph, 4]: points on the unit sphere and weights (sum 4 pi); exact for polynomials of
    degree <= min(2 nt - 1, nph - 1) = 17."""
    x, w = np.polynomial.legendre.leggauss(nt)
    ph = 2.0 * np.pi * np.arange(nph) / nph
    pts = [[math.sqrt(1 - ct * ct) * math.cos(p), math.sqrt(1 - ct * ct) * math.sin(p), ct, wt * 2 * math.pi / nph]
           for ct, wt in zip(x, w) for p in ph]
    return np.array(pts)


def radial_rule(n: int = 140):
    x, w = np.polynomial.legendre.leggauss(n)
    return (x + 1) / 2, w / 2


def _sphere_moment(a, b, c):
    """int x^a y^b z^c dOmega over the unit sphere (closed form)."""
    if a % 2 or b % 2 or c % 2:
        return 0.0
    g = math.gamma
    return 2 * g((a + 1) / 2) * g((b + 1) / 2) * g((c + 1) / 2) / g((a + b + c + 3) / 2)


def test_angular_rule_is_exact_to_degree_17():
    ang = angular_rule()
    for a in range(18):
        for b in range(18 - a):
            for c in range(18 - a - b):
                q = np.sum(ang[:, 3] * ang[:, 0] ** a * ang[:, 1] ** b * ang[:, 2] ** c)
                assert abs(q - _sphere_moment(a, b, c)) < 1e-13, (a, b, c)


def _pair_systems(orb_rads, proj_rads, tau_I, tau_J, cell=30.0):
    sp = _species(orb_rads)
    spp = _species(proj_rads)
    pos = [tau_I, tau_J]
    sysm = _system(np.eye(3) * cell, pos, [0, 0], [sp], (8, 8, 8))
    sysp = _system(np.eye(3) * cell, pos, [0, 0], [spp], (8, 8, 8))
    return Oracle(sysm, analytic=True), Oracle(sysp, analytic=True)


def test_s_type_with_phase_is_the_closed_form():
    """beta = e^{-6 x^2} Y00 at tau_I, phi = e^{-0.8 x^2} Y00 at tau_J: the integral of the Gaussian
    product K e^{-p |r - P|^2} times e^{-i A.r} is K (pi/p)^{3/2} e^{-|A|^2 / 4p} e^{-i A.P}."""
    tI, tJ = np.array([3.0, 4.0, 5.0]), np.array([5.5, 3.2, 6.1])
    o, op = _pair_systems([_gauss_radial(0, 0.8, 7.5)], [_gauss_radial(0, 6.0, 2.5)], tI, tJ)
    A = np.array([0.3, -0.2, 0.15])
    got = o.psibeta(op, A, 0, 1, radial_rule(), angular_rule())[0, 0]
    a, b = 6.0, 0.8
    p = a + b
    P = (a * tI + b * tJ) / p
    K = math.exp(-a * b * np.sum((tI - tJ) ** 2) / p)
    ref = K * (math.pi / p) ** 1.5 * math.exp(-A @ A / (4 * p)) * np.exp(-1j * (A @ P)) / (4 * math.pi)
    assert abs(got - ref) <= 1e-11 * abs(ref)


def test_p_type_with_phase_is_the_closed_form():
    """beta = (r - tau_I)_c e^{-6 |r - tau_I|^2} (real solid harmonic, l = 1), phi = e^{-0.8 x^2} Y00 at
    tau_J: with the Gaussian product K e^{-p |r - P|^2}, the integral of (r - tau_I)_c times it and
    e^{-i A.r} is K (pi/p)^{3/2} e^{-|A|^2 / 4p} e^{-i A.P} [(P - tau_I)_c - i A_c / 2p] (the moment
    from the derivative of the s-type result in A); a wrong phase centre or sign for l > 0 fails."""
    tI, tJ = np.array([3.0, 4.0, 5.0]), np.array([4.1, 5.3, 3.9])
    o, op = _pair_systems([_gauss_radial(0, 0.8, 7.5)], [_gauss_radial(1, 6.0, 2.5)], tI, tJ)
    A = np.array([0.45, -0.3, 0.6])
    got = o.psibeta(op, A, 0, 1, radial_rule(), angular_rule())[:, 0]
    a, b = 6.0, 0.8
    p = a + b
    P = (a * tI + b * tJ) / p
    K = math.exp(-a * b * np.sum((tI - tJ) ** 2) / p)
    F = K * (math.pi / p) ** 1.5 * math.exp(-A @ A / (4 * p)) * np.exp(-1j * (A @ P)) / math.sqrt(4 * math.pi)
    ref = np.zeros(3, dtype=np.complex128)
    for m, poly in enumerate(_SOLID[1]):
        for e, coef in poly.items():
            c = e.index(1)
            ref[m] += coef * F * ((P - tI)[c] - 0.5j * A[c] / p)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    assert np.abs(ref.imag).max() > 1e-3 * np.abs(ref).max()  # the field term is not negligible


def test_zero_field_is_the_two_centre_overlap():
    """A = 0: a p-type projector against s and d orbitals equals the two-centre Gaussian overlap
    (product theorem with the real solid harmonics, the same Y_lm convention)."""
    tI, tJ = np.array([10.0, 11.0, 9.0]), np.array([11.3, 9.6, 10.8])
    orb = [_gauss_radial(0, 0.8, 7.5), _gauss_radial(2, 0.7, 7.5)]
    prj = [_gauss_radial(1, 5.0, 3.0)]
    o, op = _pair_systems(orb, prj, tI, tJ)
    got = o.psibeta(op, np.zeros(3), 0, 1, radial_rule(), angular_rule())
    rows = [(tI, 5.0, poly) for poly in _SOLID[1]]
    cols = [(tJ, rad.alpha, poly) for rad in orb for poly in _SOLID[rad.l]]
    ref = np.zeros((len(rows), len(cols)))
    for i, (Ac, a, pa) in enumerate(rows):
        for j, (Bc, b, pb) in enumerate(cols):
            ref[i, j] = sum(ca * cb * np.prod([_overlap_1d(ea[c], eb[c], a, b, Ac[c], Bc[c]) for c in range(3)])
                            for ea, ca in pa.items() for eb, cb in pb.items())
    assert np.abs(got.imag).max() == 0.0
    assert np.abs(got.real - ref).max() <= 1e-10 * np.abs(ref).max()


def _si_with_projectors(shift=np.zeros(3)):
    w = inputs.config_workload("si8_g48")
    s = w.system
    pos = np.asarray(s.pos) + shift
    sysm = inputs.System(cell=s.cell, pos=pos, species=s.species, sp=s.sp, grid=s.grid)
    sysp = inputs.System(cell=s.cell, pos=pos, species=s.species, sp=[inputs.si_projectors()], grid=s.grid)
    return Oracle(sysm), Oracle(sysp)


def test_translation_multiplies_by_the_phase():
    """Moving every atom by t moves the grid with them: P(A) picks up e^{-i A.t}."""
    A = np.array([0.2, 0.1, -0.3])
    t = np.array([0.37, -0.81, 1.23])
    o0, p0 = _si_with_projectors()
    o1, p1 = _si_with_projectors(t)
    for I, J in [(0, 0), (0, 5), (3, 1)]:
        a = o0.psibeta(p0, A, I, J, radial_rule(), angular_rule())
        b = o1.psibeta(p1, A, I, J, radial_rule(), angular_rule())
        assert np.abs(b - a * np.exp(-1j * (A @ t))).max() <= 1e-13 * np.abs(a).max()


def test_opposite_field_is_the_conjugate():
    A = np.array([0.2, 0.1, -0.3])
    o, p = _si_with_projectors()
    a = o.psibeta(p, A, 2, 6, radial_rule(), angular_rule())
    b = o.psibeta(p, -A, 2, 6, radial_rule(), angular_rule())
    assert np.abs(b - a.conj()).max() <= 1e-15 * np.abs(a).max()
    assert np.abs(a).max() > 1e-4
