"""Pins for the oracle's restricted modes, which the larger GPU parity tests compare against:
the grid-point index lists of the density, local-H and force loops, the atom mask of the force
loop, and the single-block local-H routine.

Each restricted mode is checked against something fixed elsewhere: a brute-force evaluation from
scipy's Hermite spline and spherical harmonics (the same construction test_oracle_pins uses for
the full passes), or a full pass whose potential is zeroed outside the index list (the local-H sum
and the force are linear in V, and a point with V = 0 contributes nothing), so that an index
off-by-one, a point skipped by the atom-mask shortcut or a transposed block cannot pass.
Paper: the density, local-potential and local-Pulay-force sums of Sec. 3.3.1.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2603_21835_gb300 import inputs
from tests.test_oracle_pins import _brute_phi, _system


@pytest.fixture(scope="module")
def two_atoms():
    """Two Si atoms in the cubic cell (10^3 grid), a non-symmetric D and a random V."""
    w = inputs.si_workload((1, 1, 1), (10, 10, 10), seed=4)
    sysm = _system(w.system.cell, w.system.pos[[0, 4]] + 0.03, [0, 0], w.system.sp, (10, 10, 10))
    o = Oracle(sysm)
    rng = np.random.default_rng(21)
    C = rng.normal(size=(o.norb, 5))
    D = C @ C.T + 0.1 * rng.normal(size=(o.norb, o.norb))
    V = rng.normal(size=o.ngrid)
    pts = inputs.grid_points(sysm.cell, sysm.grid).reshape(-1, 3)
    Phi = _brute_phi(sysm, pts)
    idx = np.sort(rng.choice(o.ngrid, 137, replace=False))
    return sysm, o, D, V, pts, Phi, idx


def test_rho_on_index_list_equals_brute_force(two_atoms):
    _, o, D, _, _, Phi, idx = two_atoms
    ref = np.einsum("gm,mn,gn->g", Phi[idx], D, Phi[idx])
    got = o.rho(D, idx)
    assert got.shape == idx.shape
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    # and it is the full pass read at those points (an index mix-up would permute values)
    np.testing.assert_allclose(got, o.rho(D).reshape(-1)[idx], rtol=0, atol=1e-14 * np.abs(ref).max())


def test_vlocal_on_index_list_equals_brute_force(two_atoms):
    sysm, o, _, V, _, Phi, idx = two_atoms
    wgt = abs(np.linalg.det(sysm.cell)) / o.ngrid
    ref = wgt * (Phi[idx] * V[idx, None]).T @ Phi[idx]
    got = o.vlocal(V, idx)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    Vm = np.zeros_like(V)
    Vm[idx] = V[idx]
    np.testing.assert_allclose(got, o.vlocal(Vm), rtol=0, atol=1e-13 * np.abs(ref).max())


def test_force_on_index_list_equals_masked_potential(two_atoms):
    _, o, D, V, _, _, idx = two_atoms
    Vm = np.zeros_like(V)
    Vm[idx] = V[idx]
    F_idx = o.force(D, V, idx=idx)
    F_masked = o.force(D, Vm)
    assert np.abs(F_masked).max() > 0
    np.testing.assert_allclose(F_idx, F_masked, rtol=0, atol=1e-13 * np.abs(F_masked).max())


@pytest.fixture(scope="module")
def spread_cell():
    """Eight displaced Si atoms at 16^3: several atoms' supports leave points uncovered, so the
    atom-mask shortcut skips points."""
    w = inputs.si_workload((1, 1, 1), (16, 16, 16), seed=5, disp_sigma=0.1)
    sp = inputs.si_species(rc=3.5)
    sysm = _system(w.system.cell, w.system.pos, w.system.species, [sp], w.system.grid)
    o = Oracle(sysm)
    rng = np.random.default_rng(22)
    C = rng.normal(size=(o.norb, 12)) / 4
    return sysm, o, C @ C.T, rng.normal(size=o.ngrid)


def test_force_atom_mask_equals_full_force_rows(spread_cell):
    sysm, o, D, V = spread_cell
    F = o.force(D, V)
    S = np.array([1, 4, 6])
    Fs = o.force(D, V, atoms=S)
    # some points are covered by no selected atom (the shortcut is exercised)
    pts = inputs.grid_points(sysm.cell, sysm.grid).reshape(-1, 3)
    phi = o.phi_points(pts, grad=False)
    off = o.atom_offsets()
    cov = np.zeros(pts.shape[0], bool)
    for a in S:
        cov |= np.abs(phi[:, off[a]:off[a + 1]]).max(1) > 0
    assert (~cov).sum() > 0
    np.testing.assert_allclose(Fs[S], F[S], rtol=0, atol=1e-13 * np.abs(F).max())
    others = np.setdiff1d(np.arange(o.natoms), S)
    assert np.all(Fs[others] == 0.0)


def test_vlocal_block_is_the_slice_of_the_dense_pass(spread_cell):
    _, o, _, V = spread_cell
    H = o.vlocal(V)
    off = o.atom_offsets()
    for I, J in ((0, 0), (2, 5), (5, 2), (7, 3)):
        blk = o.vlocal_block(V, I, J)
        ref = H[off[I]:off[I + 1], off[J]:off[J + 1]]
        np.testing.assert_allclose(blk, ref, rtol=0, atol=1e-13 * np.abs(H).max())
