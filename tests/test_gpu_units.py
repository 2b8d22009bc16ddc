"""Unit checks of two hot-path steps on the GPU, through the library's diagnostic entry points.

1. The device grid-brick -> atom neighbour lists (the paper's BigGrid neighbour relation, Sec. 3.3.1,
   Fig. 2) against a host brute force: every lattice image of every atom whose support sphere strictly
   contains a grid point of the brick.  Exact set equality per brick (entries within 1e-9 of the
   support boundary may go either way: the device and the host form r^2 in different orders).
2. The orbital evaluators (Eqs. 1-2: cubic-Hermite radial times real Y_lm, summed over the images)
   and their gradients against the oracle at the edge radii: on the atom (r = 0), next to it, at
   Hermite knots and between them, just inside and just outside the support radius, and at random
   points.  The float64 evaluator to 1e-13 of the largest value; the tensor-core path's float32
   evaluator to 2e-6 (values) and 4e-6 (gradients) of the largest value.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2603_21835_gb300 import inputs

pytestmark = pytest.mark.gpu

BI, BJ, BK = 4, 4, 8


def _brute_lists(system):
    """Per brick: {(atom, image n1, n2, n3): min over the brick's points of |r - tau - R|^2 - rc^2}
    for the images with some point strictly inside (value < 0), plus the near-boundary images."""
    cell = np.asarray(system.cell, float)
    n = np.array(system.grid)
    nb = -(-n // np.array([BI, BJ, BK]))
    ii, jj, kk = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    frac = np.stack([ii / n[0], jj / n[1], kk / n[2]], -1).reshape(-1, 3)
    pts = frac @ cell
    bidx = (((ii // BI) * nb[1] + jj // BJ) * nb[2] + kk // BK).reshape(-1)
    inv = np.linalg.inv(cell)
    out = [dict() for _ in range(int(np.prod(nb)))]
    for a in range(system.natoms):
        rc = system.sp[system.species[a]].rcut
        u = (pts - system.pos[a]) @ inv
        reach = rc * np.linalg.norm(inv, axis=0)
        lo = np.floor(u.min(0) - reach).astype(int)
        hi = np.ceil(u.max(0) + reach).astype(int)
        for n0 in range(lo[0], hi[0] + 1):
            for n1 in range(lo[1], hi[1] + 1):
                for n2 in range(lo[2], hi[2] + 1):
                    T = system.pos[a] + np.array([n0, n1, n2]) @ cell
                    m = np.einsum("ij,ij->i", pts - T, pts - T) - rc * rc
                    near = m < 1e-9
                    if not near.any():
                        continue
                    mins = np.full(len(out), np.inf)
                    np.minimum.at(mins, bidx[near], m[near])
                    for b in np.flatnonzero(np.isfinite(mins)):
                        out[b][(a, n0, n1, n2)] = mins[b]
    return out


@pytest.mark.parametrize("case", ["si8_g48", "fcc_ragged", "water"])
def test_neighbour_lists_match_brute_force(case):
    from paper_2603_21835_gb300 import gint as G

    if case == "si8_g48":
        system = inputs.config_workload("si8_g48").system
    elif case == "fcc_ragged":  # primitive fcc cell (images fold), grid not a multiple of the brick
        a = inputs.SI_A
        cell = np.array([[0, a / 2, a / 2], [a / 2, 0, a / 2], [a / 2, a / 2, 0]])
        system = inputs.System(cell=cell, pos=np.array([[0.0, 0.0, 0.0], [a / 4, a / 4, a / 4]]) + 0.031,
                               species=np.zeros(2, np.int32), sp=[inputs.si_species()], grid=(21, 18, 27))
    else:  # two species, vacuum bricks
        system = inputs.h2o_workload(3, seed=5, box=18.0, grid=(36, 36, 40)).system
    g = G.Gint(system)
    b_off, slot_atom, slot_ent, epos = g.brick_lists()
    ref = _brute_lists(system)
    assert len(b_off) == len(ref) + 1
    inv = np.linalg.inv(np.asarray(system.cell, float))
    nent = 0
    for b, want in enumerate(ref):
        got = {}
        atoms = slot_atom[b_off[b]:b_off[b + 1]]
        assert np.all(np.diff(atoms) > 0), "slots of a brick are distinct and sorted by atom"
        for s in range(b_off[b], b_off[b + 1]):
            a = int(slot_atom[s])
            for e in range(slot_ent[s], slot_ent[s + 1]):
                nvec = (epos[e] - system.pos[a]) @ inv
                key = (a,) + tuple(int(x) for x in np.rint(nvec))
                assert np.abs(nvec - np.rint(nvec)).max() < 1e-9  # an exact lattice image
                assert key not in got
                got[key] = True
                nent += 1
        sure = {k for k, v in want.items() if v < -1e-9}
        maybe = {k for k, v in want.items() if -1e-9 <= v < 1e-9}
        assert sure <= set(got), (b, sorted(sure - set(got)))
        assert set(got) <= sure | maybe, (b, sorted(set(got) - sure - maybe))
    assert nent == len(epos)
    g.close()


def _edge_points(system, rng):
    """Points around atom 0 at the edge radii of its radial tables, random directions."""
    rad = system.sp[system.species[0]].radials[0]
    rc, dr = rad.rc, rad.dr
    radii = [0.0, 1e-9, 1e-6, dr, 10 * dr, 10.5 * dr, 350 * dr, 350.25 * dr, rc - 3 * dr, rc - 1e-9, rc + 1e-9,
             rc - 0.5 * dr]
    d = rng.normal(size=(len(radii), 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pts = system.pos[0] + np.array(radii)[:, None] * d
    pts[0] = system.pos[0]
    cell = np.asarray(system.cell, float)
    pts = np.concatenate([pts, rng.uniform(0, 1, size=(40, 3)) @ cell])
    return pts


@pytest.mark.parametrize("prec,tol,gtol", [("fp64", 1e-13, 1e-13), ("f16x3", 2e-6, 4e-6)])
def test_orbital_evaluators_match_oracle_at_edge_radii(prec, tol, gtol):
    from paper_2603_21835_gb300 import gint as G

    w = inputs.si_workload((1, 1, 1), (24, 24, 24), seed=3, disp_sigma=0.05)
    rng = np.random.default_rng(17)
    pts = _edge_points(w.system, rng)
    o = Oracle(w.system)
    ref_phi, ref_grad = o.phi_points(pts)
    g = G.Gint(w.system)
    phi, grad = g.orbitals(pts, G.PRECISIONS[prec])
    ep = np.abs(phi - ref_phi).max() / np.abs(ref_phi).max()
    eg = np.abs(grad - ref_grad).max() / np.abs(ref_grad).max()
    print(prec, "phi", ep, "grad", eg)
    assert ep <= tol and eg <= gtol
    # on the atom: only the s orbitals of atom 0 are non-zero among its own (the reading for r = 0)
    off = o.atom_offsets()
    own = phi[0, off[0]:off[1]]
    l_of = np.concatenate([[r.l] * (2 * r.l + 1) for r in w.system.sp[0].radials])
    assert np.all(np.abs(ref_phi[0, off[0]:off[1]][l_of > 0]) == 0.0)
    assert np.abs(own[l_of > 0]).max() <= tol * np.abs(ref_phi).max()
    g.close()
