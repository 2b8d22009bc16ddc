"""Host-side pins of the synthetic input recipe (no method arithmetic): the diamond geometry and atom
order, the periodic-Gaussian V against a brute-force image sum, seeded determinism, wrapped
displacements, the rigid water clusters and their spacing, and the serving mix."""
import itertools
import math

import numpy as np

from paper_2603_21835_gb300 import inputs


def test_diamond_supercell_order_and_bonds():
    cell, pos = inputs.si_supercell((1, 2, 3))
    a = inputs.SI_A
    assert pos.shape == (8 * 6, 3)
    # cell (i, j, k) outer with k fastest, basis inner
    for (i, j, k), b in [((0, 1, 2), 4), ((0, 0, 1), 0), ((0, 1, 0), 7)]:
        idx = 8 * (i * 6 + j * 3 + k) + b
        ref = (np.array([i, j, k]) + np.array(inputs.DIAMOND_BASIS[b])) * a
        assert np.abs(pos[idx] - ref).max() < 1e-12
    # four nearest neighbours at a sqrt(3) / 4 (minimum image), the next shell at a / sqrt(2)
    inv = np.linalg.inv(cell)
    for n in range(len(pos)):
        d = (pos - pos[n]) @ inv
        d -= np.round(d)
        r = np.sort(np.linalg.norm(d @ cell, axis=1))[1:]
        assert np.allclose(r[:4], a * math.sqrt(3) / 4, atol=1e-9)
        assert abs(r[4] - a / math.sqrt(2)) < 1e-9


def test_periodic_gaussians_match_the_image_sum():
    """The orthorhombic path factorises the Gaussian per axis; it equals the 3-D sum over
    R in [-2, 2]^3 written out."""
    cell = np.diag([7.0, 8.0, 9.0])
    grid = (6, 5, 4)
    rng = np.random.default_rng(3)
    c, s, A = rng.random((3, 3)), rng.uniform(1, 3, 3), rng.normal(0, 0.5, 3)
    V = inputs.periodic_gaussians_V(cell, grid, c, s, A)
    pts = inputs.grid_points(cell, grid)
    ref = np.zeros(len(pts))
    for cc, ss, aa in zip(c, s, A):
        for n in itertools.product(range(-2, 3), repeat=3):
            d = pts - cc @ cell - np.array(n) @ cell
            ref += aa * np.exp(-(d * d).sum(1) / (2 * ss * ss))
    assert np.abs(V.reshape(-1) - ref).max() <= 1e-13 * np.abs(ref).max()


def test_workloads_are_seeded_and_D_is_psd():
    a, b = inputs.config_workload("si8_g48"), inputs.config_workload("si8_g48")
    assert np.array_equal(a.V, b.V) and np.array_equal(a.C, b.C) and np.array_equal(a.D, b.D)
    assert a.V.shape == (48, 48, 48) and a.C.shape == (104, 16)
    assert np.array_equal(a.D, a.D.T)
    assert np.linalg.eigvalsh(a.D).min() > -1e-12 * np.abs(a.D).max()


def test_displacements_are_wrapped_and_of_the_stated_width():
    w = inputs.config_workload("si64_g96_d", dense_D=False)
    cell = w.system.cell
    frac = w.system.pos @ np.linalg.inv(cell)
    assert (frac >= 0).all() and (frac < 1).all()
    _, pos0 = inputs.si_supercell((2, 2, 2))
    d = (w.system.pos - pos0) @ np.linalg.inv(cell)
    d -= np.round(d)
    d = d @ cell
    assert 0.08 < d.std() < 0.12  # N(0, 0.1) Bohr per component, 192 samples


def test_water_clusters_are_rigid_and_spaced():
    pool = inputs.serving_pool()
    _, water = inputs.serving_kinds()
    for k, nmol in zip(water, inputs.SERVING_H2O):
        s = pool[k]
        assert s.pos.shape == (3 * nmol, 3)
        names = [s.sp[t].name for t in s.species]
        assert names == ["O", "H", "H"] * nmol
        m = s.pos.reshape(nmol, 3, 3)
        O, H1, H2 = m[:, 0], m[:, 1], m[:, 2]
        assert np.allclose(np.linalg.norm(H1 - O, axis=1), inputs.OH_BOND)
        assert np.allclose(np.linalg.norm(H2 - O, axis=1), inputs.OH_BOND)
        ang = np.degrees(np.arccos(((H1 - O) * (H2 - O)).sum(1) / inputs.OH_BOND ** 2))
        assert np.allclose(ang, 104.5)
        dOO = np.linalg.norm(O[:, None] - O[None], axis=2) + 1e9 * np.eye(nmol)
        assert dOO.min() >= 4.5
        Rs = (3.0 * nmol / (4.0 * math.pi * 0.00495)) ** (1.0 / 3.0)
        assert (np.linalg.norm(O - 15.0, axis=1) <= Rs + 1e-12).all()


def test_serving_mix():
    si, water = inputs.serving_kinds()
    pool = inputs.serving_pool()
    assert len(si) == 10 and len(water) == 4
    assert sorted(pool[k].natoms for k in si) == sorted(8 * a * b * c for a, b, c in inputs.SERVING_SI_CELLS)
    req = inputs.serving_requests(256, seed=1)
    assert req == inputs.serving_requests(256, seed=1)
    frac_si = np.mean([r in si for r in req])
    assert 0.4 < frac_si < 0.6
