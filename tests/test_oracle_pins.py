"""Pins for the FP64 oracle against closed forms, library routines, invariants and
finite differences.  Nothing here compares the oracle with itself retyped: each
test checks it against something the mathematics or an independent library fixes.

Paper references: orbital form Eq. 1, Gamma-point Bloch sum Eq. 2, and the
density / local-Hamiltonian / local-Pulay-force formulas of Sec. 3.3.1.
"""
import math

import numpy as np
import pytest
from scipy.interpolate import CubicHermiteSpline
from scipy.special import gamma, sph_harm_y

from oracle.oracle import Oracle
from paper_2603_21835_gb300 import inputs


# ----------------------------------------------------------------------------- helpers
def _species(rads, name="X"):
    return inputs.Species(name=name, radials=rads)


def _gauss_radial(l, alpha, rc, dr=0.01):
    """Radial record for the oracle's analytic mode (table unused but kept valid)."""
    return inputs.make_radial(l, alpha, rc, dr)


def _system(cell, pos, species, sp, grid):
    return inputs.System(cell=np.asarray(cell, float), pos=np.asarray(pos, float),
                         species=np.asarray(species, np.int32), sp=sp, grid=tuple(grid))


def _real_ylm_scipy(l, pts):
    """Real orthonormal Y_lm (no Condon-Shortley sign), order m=0,+1,-1,+2,-2, from scipy's complex Y."""
    r = np.linalg.norm(pts, axis=1)
    theta = np.arccos(np.clip(pts[:, 2] / r, -1, 1))
    ph = np.arctan2(pts[:, 1], pts[:, 0])
    out = [np.real(sph_harm_y(l, 0, theta, ph))]
    for m in range(1, l + 1):
        y = sph_harm_y(l, m, theta, ph)  # includes (-1)^m
        out.append(math.sqrt(2) * (-1) ** m * np.real(y))
        out.append(math.sqrt(2) * (-1) ** m * np.imag(y))
    return np.stack(out, axis=1)


def _brute_phi(system, pts):
    """Periodised orbitals by brute force: scipy CubicHermiteSpline radials x scipy real Y_lm,
    summed over an explicit block of lattice images."""
    cell = system.cell
    nimg = 3
    rng = np.arange(-nimg, nimg + 1)
    shifts = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3) @ cell
    cols = []
    for a in range(system.natoms):
        sp = system.sp[system.species[a]]
        blocks = [np.zeros((pts.shape[0], 2 * r.l + 1)) for r in sp.radials]
        for R in shifts:
            d = pts - system.pos[a] - R
            r = np.linalg.norm(d, axis=1)
            for k, rad in enumerate(sp.radials):
                inside = r < rad.rc
                if not inside.any():
                    continue
                knots = np.arange(rad.npts) * rad.dr
                spl = CubicHermiteSpline(knots, rad.f, rad.df)
                f = np.where(inside, spl(np.minimum(r, knots[-1])), 0.0)
                dd = d[inside]
                Y = np.zeros((pts.shape[0], 2 * rad.l + 1))
                rs = np.linalg.norm(dd, axis=1)
                ok = rs > 1e-12
                Yin = np.zeros((dd.shape[0], 2 * rad.l + 1))
                if ok.any():
                    Yin[ok] = _real_ylm_scipy(rad.l, dd[ok])
                if rad.l == 0:
                    Yin[~ok] = 0.5 / math.sqrt(math.pi)
                Y[inside] = Yin
                blocks[k] += f[:, None] * Y
        cols.extend(blocks)
    return np.concatenate(cols, axis=1)


# ----------------------------------------------------------------------------- radial interpolation
def test_hermite_reproduces_cubics_exactly():
    """A cubic Hermite interpolant is exact for cubic polynomials (f and f' given exactly)."""
    c = np.array([0.7, -0.3, 0.05, -0.002])
    rc, dr = 5.0, 0.05
    knots = np.arange(int(round(rc / dr)) + 1) * dr
    f = c[0] + c[1] * knots + c[2] * knots**2 + c[3] * knots**3
    df = c[1] + 2 * c[2] * knots + 3 * c[3] * knots**2
    rad0 = inputs.Radial(l=0, alpha=0.0, rc=rc, dr=dr, f=f, df=df)
    rad1 = inputs.Radial(l=1, alpha=0.0, rc=rc, dr=dr, f=f, df=df)
    sysm = _system(np.eye(3) * 30, [[15, 15, 15]], [0], [_species([rad0, rad1])], (8, 8, 8))
    o = Oracle(sysm)
    r = np.random.default_rng(3).uniform(0.01, rc - dr, 200)
    pts = np.stack([np.full_like(r, 15), np.full_like(r, 15), 15 + r], 1)  # along +z
    phi, g = o.phi_points(pts)
    fr = c[0] + c[1] * r + c[2] * r**2 + c[3] * r**3
    dfr = c[1] + 2 * c[2] * r + 3 * c[3] * r**2
    y00, y1 = 0.5 / math.sqrt(math.pi), math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(phi[:, 0], fr * y00, rtol=0, atol=1e-14)
    np.testing.assert_allclose(phi[:, 1], fr * y1, rtol=0, atol=1e-14)  # m=0 ~ z
    np.testing.assert_allclose(phi[:, 2:4], 0, atol=1e-15)  # x, y components vanish on the z axis
    np.testing.assert_allclose(g[:, 0, 2], dfr * y00, atol=1e-13)


def test_radial_interpolation_error_bound():
    """|f - H f| <= dr^4 max|f''''| / 384 (textbook bound for cubic Hermite)."""
    sp = inputs.si_species()
    sysm = _system(np.eye(3) * 40, [[20, 20, 20]], [0], [sp], (8, 8, 8))
    o = Oracle(sysm)
    rng = np.random.default_rng(5)
    r = rng.uniform(0.0, 6.99, 400)
    dirs = rng.normal(size=(400, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    pts = 20 + r[:, None] * dirs
    phi = o.phi_points(pts, grad=False)
    col = 0
    for rad in sp.radials:
        fe, _ = inputs.radial_shape(r, rad.l, rad.alpha, rad.rc)
        Y = _real_ylm_scipy(rad.l, r[:, None] * dirs)
        exact = fe[:, None] * Y
        fine = np.linspace(0, rad.rc, 200001)
        f4 = np.gradient(np.gradient(np.gradient(np.gradient(inputs.radial_shape(fine, rad.l, rad.alpha, rad.rc)[0], fine), fine), fine), fine)
        bound = rad.dr**4 * np.abs(f4).max() / 384 * 1.01
        nm = 2 * rad.l + 1
        assert np.abs(phi[:, col:col + nm] - exact).max() <= bound
        col += nm


# ----------------------------------------------------------------------------- angular part and gradients
def test_orbitals_match_scipy_spherical_harmonics():
    sp = inputs.si_species()
    sysm = _system(np.eye(3) * 40, [[20, 20, 20]], [0], [sp], (8, 8, 8))
    o = Oracle(sysm)
    rng = np.random.default_rng(11)
    pts = 20 + rng.uniform(-5, 5, (300, 3))
    phi = o.phi_points(pts, grad=False)
    ref = _brute_phi(sysm, pts)
    np.testing.assert_allclose(phi, ref, rtol=0, atol=1e-13)


def test_gradients_match_central_differences():
    sp = inputs.si_species()
    cell = np.array([[0, 5.13, 5.13], [5.13, 0, 5.13], [5.13, 5.13, 0]])  # fcc primitive: images overlap
    sysm = _system(cell, [[0.1, 0.2, 0.3], [2.6, 2.5, 2.7]], [0, 0], [sp], (8, 8, 8))
    o = Oracle(sysm)
    rng = np.random.default_rng(2)
    pts = rng.uniform(-3, 6, (60, 3))
    _, g = o.phi_points(pts)
    h = 1e-5
    fd = np.zeros_like(g)
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        fd[:, :, c] = (o.phi_points(pts + e, grad=False) - o.phi_points(pts - e, grad=False)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=0, atol=2e-8)


def test_grid_point_on_atom_is_the_continuous_limit():
    """At |d| = 0 the rule (phi_s = f(0) Y00, grad phi_p = f'(0) sqrt(3/4pi) e_m, others 0)
    equals the limit of the general formula approached from a nearby point."""
    sp = inputs.si_species()
    sysm = _system(np.eye(3) * 40, [[20, 20, 20]], [0], [sp], (8, 8, 8))
    o = Oracle(sysm)
    p0, g0 = o.phi_points(np.array([[20.0, 20.0, 20.0]]))
    for d in ([1e-7, 0, 0], [0, -1e-7, 0], [0, 0, 1e-7], [6e-8, -5e-8, 4e-8]):
        p1, g1 = o.phi_points(np.array([[20.0, 20.0, 20.0]]) + np.array(d))
        np.testing.assert_allclose(p0, p1, atol=1e-6)
        np.testing.assert_allclose(g0, g1, atol=1e-5)
    assert p0[0, 0] == pytest.approx(sp.radials[0].f[0] * 0.5 / math.sqrt(math.pi), rel=1e-15)
    assert abs(g0[0, 2, 2]) > 0.1 and abs(g0[0, 3, 0]) > 0.1 and abs(g0[0, 4, 1]) > 0.1  # p zeta0: z, x, y


# ----------------------------------------------------------------------------- closed-form Gaussian overlaps
_SOLID = {  # real solid harmonics r^l Y_lm as {monomial exponent: coefficient}, m = 0,+1,-1,+2,-2
    0: [{(0, 0, 0): 0.5 / math.sqrt(math.pi)}],
    1: [{(0, 0, 1): math.sqrt(3 / (4 * math.pi))}, {(1, 0, 0): math.sqrt(3 / (4 * math.pi))},
        {(0, 1, 0): math.sqrt(3 / (4 * math.pi))}],
    2: [{(0, 0, 2): 2 * math.sqrt(5 / (16 * math.pi)), (2, 0, 0): -math.sqrt(5 / (16 * math.pi)),
         (0, 2, 0): -math.sqrt(5 / (16 * math.pi))},
        {(1, 0, 1): math.sqrt(15 / (4 * math.pi))}, {(0, 1, 1): math.sqrt(15 / (4 * math.pi))},
        {(2, 0, 0): math.sqrt(15 / (16 * math.pi)), (0, 2, 0): -math.sqrt(15 / (16 * math.pi))},
        {(1, 1, 0): math.sqrt(15 / (4 * math.pi))}],
}


def _overlap_1d(i, j, a, b, A, B):
    """int (x-A)^i (x-B)^j exp(-a(x-A)^2 - b(x-B)^2) dx by the Gaussian product theorem."""
    p = a + b
    P = (a * A + b * B) / p
    K = math.exp(-a * b * (A - B) ** 2 / p)
    tot = 0.0
    for s in range(i + 1):
        for t in range(j + 1):
            k = s + t
            if k % 2:
                continue
            M = gamma((k + 1) / 2) / p ** ((k + 1) / 2)
            tot += math.comb(i, s) * math.comb(j, t) * (P - A) ** (i - s) * (P - B) ** (j - t) * M
    return K * tot


def _gaussian_overlap_matrix(system, nimg=3):
    """S_{mu nu} = sum_R int phi_mu(r - tau_I) phi_nu(r - tau_J - R) dr for r^l e^{-alpha r^2} Y_lm."""
    orbs = []
    for a in range(system.natoms):
        for rad in system.sp[system.species[a]].radials:
            for poly in _SOLID[rad.l]:
                orbs.append((system.pos[a], rad.alpha, poly))
    n = len(orbs)
    rng = np.arange(-nimg, nimg + 1)
    shifts = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3) @ system.cell
    S = np.zeros((n, n))
    for i, (A, a, pa) in enumerate(orbs):
        for j, (B0, b, pb) in enumerate(orbs):
            acc = 0.0
            for R in shifts:
                B = B0 + R
                if np.linalg.norm(A - B) > 12:
                    continue
                for ea, ca in pa.items():
                    for eb, cb in pb.items():
                        acc += ca * cb * np.prod([_overlap_1d(ea[c], eb[c], a, b, A[c], B[c]) for c in range(3)])
            S[i, j] = acc
    return S


@pytest.mark.parametrize("cellkind", ["cubic", "triclinic"])
def test_grid_overlap_equals_closed_form_gaussian_overlap(cellkind):
    """V = 1: H_grid is the overlap S; for Gaussian-type NAOs (cutoff where e^{-alpha rc^2} < 1e-17)
    the periodic trapezoid sum converges spectrally to the lattice-summed closed form."""
    rc = 7.5
    sp = _species([_gauss_radial(0, 0.8, rc), _gauss_radial(1, 1.0, rc), _gauss_radial(2, 1.2, rc),
                   _gauss_radial(0, 1.5, rc)])
    if cellkind == "cubic":
        cell = np.eye(3) * 7.0
        grid = (24, 24, 24)
    else:
        cell = np.array([[7.0, 0.0, 0.0], [1.5, 6.8, 0.0], [-1.0, 0.9, 7.2]])
        grid = (26, 26, 27)
    sysm = _system(cell, [[0.3, 1.1, 0.7], [3.9, 2.2, 4.4]], [0, 0], [sp], grid)
    o = Oracle(sysm, analytic=True)
    H = o.vlocal(np.ones(o.ngrid))
    S = _gaussian_overlap_matrix(sysm)
    assert np.abs(H - S).max() / np.abs(S).max() < 1e-13
    # the density identity against the same closed form: sum_g w rho = sum D*S
    D = np.random.default_rng(0).normal(size=S.shape)
    assert o.weight() * o.rho(D).sum() == pytest.approx(np.sum(D * S), rel=1e-10, abs=1e-10)


def test_same_centre_overlap_equals_radial_quadrature():
    """One atom, images farther apart than 2 rc: S = delta_{ll'} delta_{mm'} int R R' r^2 dr
    (angular orthonormality), the radial integral by 200-point Gauss-Legendre."""
    sp = inputs.si_species()
    L, n = 16.0, 80
    sysm = _system(np.eye(3) * L, [[8.0 + 0.013, 8.0 - 0.021, 8.0 + 0.007]], [0], [sp], (n, n, n))
    o = Oracle(sysm)
    S = o.vlocal(np.ones(o.ngrid))
    x, wq = np.polynomial.legendre.leggauss(200)
    rc = 7.0
    r = 0.5 * rc * (x + 1)
    wq = 0.5 * rc * wq
    ref = np.zeros_like(S)
    offs = []
    col = 0
    for rad in sp.radials:
        offs.append(col)
        col += 2 * rad.l + 1
    for a, ra in enumerate(sp.radials):
        for b, rb in enumerate(sp.radials):
            if ra.l != rb.l:
                continue
            fa = inputs.radial_shape(r, ra.l, ra.alpha, ra.rc)[0]
            fb = inputs.radial_shape(r, rb.l, rb.alpha, rb.rc)[0]
            val = np.sum(wq * fa * fb * r * r)
            for m in range(2 * ra.l + 1):
                ref[offs[a] + m, offs[b] + m] = val
    assert np.abs(S - ref).max() / np.abs(ref).max() < 1e-9


# ----------------------------------------------------------------------------- brute force with library routines
def test_rho_and_H_match_brute_force():
    """Tiny two-atom Si cell, 10^3 grid: oracle rho and H equal a dense numpy evaluation
    built from scipy's CubicHermiteSpline and scipy's spherical harmonics."""
    w = inputs.si_workload((1, 1, 1), (10, 10, 10), seed=4)
    sysm = _system(w.system.cell, w.system.pos[[0, 4]], [0, 0], w.system.sp, (10, 10, 10))
    o = Oracle(sysm)
    rng = np.random.default_rng(9)
    C = rng.normal(size=(o.norb, 5))
    D = C @ C.T + 0.1 * rng.normal(size=(o.norb, o.norb))  # not symmetric on purpose
    V = rng.normal(size=o.ngrid)
    pts = inputs.grid_points(sysm.cell, sysm.grid)
    Phi = _brute_phi(sysm, pts)
    wgt = abs(np.linalg.det(sysm.cell)) / o.ngrid
    rho_ref = np.einsum("gm,mn,gn->g", Phi, D, Phi)
    H_ref = wgt * (Phi * V[:, None]).T @ Phi
    np.testing.assert_allclose(o.rho(D).reshape(-1), rho_ref, rtol=0, atol=1e-12 * np.abs(rho_ref).max())
    np.testing.assert_allclose(o.vlocal(V), H_ref, rtol=0, atol=1e-12 * np.abs(H_ref).max())
    W, sn = o.count_pairs()
    # n_g by brute force: atoms with some image within rc of g
    cov = np.zeros((o.ngrid, 2), bool)
    nimg = 3
    rr = np.arange(-nimg, nimg + 1)
    shifts = np.stack(np.meshgrid(rr, rr, rr, indexing="ij"), -1).reshape(-1, 3) @ sysm.cell
    for a in range(2):
        d = pts[:, None, :] - sysm.pos[a] - shifts[None]
        cov[:, a] = (np.linalg.norm(d, axis=2) < 7.0).any(1)
    ng = cov.sum(1) * 13
    assert W == float(np.sum(ng.astype(float) ** 2)) and sn == float(ng.sum())


# ----------------------------------------------------------------------------- algebraic identities
@pytest.fixture(scope="module")
def small_si():
    w = inputs.si_workload((1, 1, 1), (24, 24, 24), seed=1, disp_sigma=0.1)
    return w, Oracle(w.system)


def test_identities(small_si):
    w, o = small_si
    V = w.V.reshape(-1)
    rho = o.rho(w.D).reshape(-1)
    S = o.vlocal(np.ones(o.ngrid))
    H = o.vlocal(V)
    wt = o.weight()
    assert wt * rho.sum() == pytest.approx(np.sum(w.D * S), rel=1e-12)  # N_e = Tr(DS)
    assert wt * np.dot(V, rho) == pytest.approx(np.sum(w.D * H), rel=1e-12)  # E = Tr(DH)
    assert np.abs(H - H.T).max() <= 1e-14 * np.abs(H).max()
    assert rho.min() >= -1e-14 * rho.max()  # D = C C^T is PSD
    # linearity in V and in D
    V2 = np.roll(V, 7)
    np.testing.assert_allclose(o.vlocal(2 * V - 0.5 * V2), 2 * H - 0.5 * o.vlocal(V2), atol=1e-13 * np.abs(H).max())
    D2 = np.eye(o.norb)
    np.testing.assert_allclose(o.rho(w.D + 3 * D2).reshape(-1), rho + 3 * o.rho(D2).reshape(-1),
                               atol=1e-12 * rho.max())


def test_translation_by_grid_vector(small_si):
    w, o = small_si
    n = np.array(w.system.grid)
    shift = np.array([3, 5, 2])
    t = (shift / n) @ w.system.cell
    moved = _system(w.system.cell, w.system.pos + t, w.system.species, w.system.sp, w.system.grid)
    o2 = Oracle(moved)
    V = w.V
    V2 = np.roll(V, shift=tuple(shift), axis=(0, 1, 2))
    rho1 = o.rho(w.D)
    rho2 = o2.rho(w.D)
    np.testing.assert_allclose(rho2, np.roll(rho1, tuple(shift), (0, 1, 2)), atol=1e-13 * rho1.max())
    H1, H2 = o.vlocal(V), o2.vlocal(V2)
    np.testing.assert_allclose(H2, H1, atol=1e-13 * np.abs(H1).max())
    F1, F2 = o.force(w.D, V), o2.force(w.D, V2)
    np.testing.assert_allclose(F2, F1, atol=1e-12 * np.abs(F1).max())


def test_constant_potential_translation_and_net_force(small_si):
    """Constant V: E = V0 * N_e; an arbitrary rigid shift changes it only at grid-aliasing level,
    and the forces sum to ~0 (same aliasing level)."""
    w, o = small_si
    V = np.full(o.ngrid, 0.7)
    E0 = o.energy(w.D, V)
    t = np.array([0.0371, -0.0523, 0.0117])
    moved = _system(w.system.cell, w.system.pos + t, w.system.species, w.system.sp, w.system.grid)
    E1 = Oracle(moved).energy(w.D, V)
    assert abs(E1 - E0) < 1e-3 * abs(E0)
    F = o.force(w.D, V)
    assert np.abs(F.sum(0)).max() < 1e-2 * np.abs(F).max()


# ----------------------------------------------------------------------------- forces by finite differences
@pytest.mark.parametrize("analytic", [False, True])
def test_forces_match_central_differences(analytic):
    rc = 7.0
    sp = inputs.si_species(rc) if not analytic else _species(
        [_gauss_radial(0, 0.8, 7.5), _gauss_radial(1, 1.0, 7.5), _gauss_radial(2, 1.2, 7.5)])
    cell = np.eye(3) * inputs.SI_A
    pos = np.array([[0.11, 0.23, -0.05], [2.5, 2.7, 2.45]])
    grid = (24, 24, 24)
    sysm = _system(cell, pos, [0, 0], [sp], grid)
    o = Oracle(sysm, analytic=analytic)
    rng = np.random.default_rng(7)
    C = rng.normal(size=(o.norb, 4)) / 4
    D = C @ C.T
    V = inputs.draw_V(np.random.default_rng(8), cell, grid).reshape(-1)
    F = o.force(D, V)
    h = 1e-4
    fd = np.zeros_like(F)
    for a in range(2):
        for c in range(3):
            for sgn in (1, -1):
                p = pos.copy()
                p[a, c] += sgn * h
                E = Oracle(_system(cell, p, [0, 0], [sp], grid), analytic=analytic).energy(D, V)
                fd[a, c] -= sgn * E / (2 * h)
    assert np.abs(F - fd).max() < 1e-8
