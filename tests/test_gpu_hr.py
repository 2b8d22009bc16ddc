"""GPU parity of the local H per lattice vector, H_IJ(R), and its Bloch sum H(k) = sum_R e^{ik.R} H(R)
(paper Sec. 2; the local-potential matrix element of Sec. 3.3.1) against the FP64 oracle on the same
seeded inputs.  Tolerance of the tensor-core F16X3 path: 1e-6 of max |H| (max-norm relative).

Two cells: the 64-atom Si supercell, where every brick sees at most one image of an atom, and the
8-atom cubic cell, where bricks see several images of one atom (folded tiles mix R): there the
handle computes H(R) on its unfolded twin (one slot per atom image), so the Gamma block (folded
tiles) and the sum of H(R) over R (unfolded tiles) come from different brick passes and agree to
the F16X3 tolerance of each, not to the bit."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2603_21835_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-6


# workload, atom pairs sampled against the oracle, tolerance of sum_R H(R) against the Gamma block
CELLS = {
    "si64_g96": ([(0, 0), (0, 1), (5, 40), (63, 2)], 1e-9),
    "si8_g48": ([(0, 0), (0, 1), (3, 5), (7, 2)], 2 * TOL),
}


@pytest.fixture(scope="module", params=sorted(CELLS))
def cell(request):
    import torch

    from paper_2603_21835_gb300 import gint as G

    w = inputs.config_workload(request.param)
    g = G.Gint(w.system)
    keys, off = g.layout_R()
    V = torch.from_numpy(np.ascontiguousarray(w.V.reshape(-1))).cuda()
    HR_dev = g.vlocal_R(V, G.F16X3)
    H = g.vlocal(V, G.F16X3).cpu().numpy()
    g.sync()
    pairs, gtol = CELLS[request.param]
    yield dict(w=w, g=g, G=G, keys=keys, off=off, HR_dev=HR_dev, HR=HR_dev.cpu().numpy(), H=H, o=Oracle(w.system),
               torch=torch, pairs=pairs, gtol=gtol, name=request.param)
    g.close()


def _block(s, q):
    I, J = s["keys"][q, :2]
    nI, nJ = s["o"]._norb_atom(I), s["o"]._norb_atom(J)
    return s["HR"][s["off"][q]:s["off"][q + 1]].reshape(nI, nJ)


def test_keys_closed_under_transposition(cell):
    s = cell
    keys = s["keys"]
    assert len(keys) > 0 and np.all(np.diff(s["off"]) > 0)
    index = {tuple(k): q for q, k in enumerate(keys)}
    assert [tuple(k) for k in keys] == sorted(index)  # sorted by (I, J, n1, n2, n3)
    hmax = np.abs(s["HR"]).max()
    for q, k in enumerate(keys):
        t = index[(k[1], k[0], -k[2], -k[3], -k[4])]
        if k[0] != k[1] or any(k[2:]):
            assert t != q and np.array_equal(_block(s, t), _block(s, q).T)  # one sum, written twice
        else:  # on-site (R = 0): symmetric to the split products' rounding
            assert np.abs(_block(s, q) - _block(s, q).T).max() <= TOL * hmax


def test_sum_over_R_is_the_gamma_block(cell):
    s = cell
    g, keys = s["g"], s["keys"]
    acc = np.zeros_like(s["H"])
    for q, k in enumerate(keys):
        p = g.block_index(int(k[0]), int(k[1]))
        assert p >= 0
        acc[g.pair_off[p]:g.pair_off[p + 1]] += s["HR"][s["off"][q]:s["off"][q + 1]]
    assert np.abs(acc - s["H"]).max() <= s["gtol"] * np.abs(s["H"]).max()


def _pair_keys(s, I, J):
    return [q for q, k in enumerate(s["keys"]) if k[0] == I and k[1] == J]


def test_sampled_blocks_match_the_oracle(cell):
    """Every R of a few atom pairs (on-site, nearest and farther neighbours) against the oracle, which
    also confirms that no overlapping image pair is missing from the key list."""
    s = cell
    hmax = np.abs(s["HR"]).max()
    for I, J in s["pairs"]:
        qs = _pair_keys(s, I, J)
        assert qs, (I, J)
        R = s["keys"][qs, 2:]
        ref, missed = s["o"].vlocal_block_R(s["w"].V, I, J, R)
        assert missed <= 1e-12 * hmax, (I, J, missed)
        for i, q in enumerate(qs):
            assert np.abs(_block(s, q) - ref[i]).max() <= TOL * hmax, (I, J, tuple(R[i]))


def test_bloch_sum(cell):
    s = cell
    g, torch = s["g"], s["torch"]
    Hk0 = g.bloch(s["HR_dev"], [0.0, 0.0, 0.0]).cpu().numpy()
    assert np.all(Hk0.imag == 0.0)
    assert np.abs(Hk0.real - s["H"]).max() <= s["gtol"] * np.abs(s["H"]).max()
    kf = np.array([0.25, 0.1, -0.3])
    Hk = g.bloch(s["HR_dev"], kf).cpu().numpy()
    g.sync()
    hmax = np.abs(s["HR"]).max()
    # Hermitian: H_JI(k) = H_IJ(k)^dagger
    for I, J in s["pairs"][1:]:
        p, t = g.block_index(I, J), g.block_index(J, I)
        nI, nJ = s["o"]._norb_atom(I), s["o"]._norb_atom(J)
        A = Hk[g.pair_off[p]:g.pair_off[p + 1]].reshape(nI, nJ)
        B = Hk[g.pair_off[t]:g.pair_off[t + 1]].reshape(nJ, nI)
        assert np.abs(B - A.conj().T).max() <= 1e-12 * hmax
    # against the oracle's H(R) summed with the phases
    for I, J in s["pairs"][1::2]:
        qs = _pair_keys(s, I, J)
        R = s["keys"][qs, 2:]
        ref, _ = s["o"].vlocal_block_R(s["w"].V, I, J, R)
        ph = np.exp(2j * np.pi * (R @ kf))
        refk = np.tensordot(ph, ref, axes=1)
        p = g.block_index(I, J)
        A = Hk[g.pair_off[p]:g.pair_off[p + 1]].reshape(refk.shape)
        assert np.abs(A - refk).max() <= len(qs) * TOL * hmax


def test_several_k_points_in_one_call(cell):
    """Nine k points (two launches of up to eight) equal nine single-k calls."""
    s = cell
    g = s["g"]
    kf = np.random.default_rng(4).uniform(-0.5, 0.5, size=(9, 3))
    many = g.bloch(s["HR_dev"], kf).cpu().numpy()
    for j in range(9):
        one = g.bloch(s["HR_dev"], kf[j]).cpu().numpy()
        assert np.array_equal(many[j], one)


def test_water_cluster_two_species():
    """Water molecules in a 20 Bohr box (O: 13 orbitals, H: 5; blocks of different shapes): every R
    of a few pairs against the oracle."""
    import torch

    from paper_2603_21835_gb300 import gint as G

    w = inputs.h2o_workload(6, seed=3, box=20.0, grid=(64, 64, 64))
    g = G.Gint(w.system)
    keys, off = g.layout_R()
    V = torch.from_numpy(np.ascontiguousarray(w.V.reshape(-1))).cuda()
    HR = g.vlocal_R(V, G.F16X3).cpu().numpy()
    g.sync()
    o = Oracle(w.system)
    hmax = np.abs(HR).max()
    for I, J in [(0, 1), (1, 2), (0, 3), (2, 2)]:
        qs = [q for q, k in enumerate(keys) if k[0] == I and k[1] == J]
        if not qs:
            continue
        R = keys[qs, 2:]
        ref, missed = o.vlocal_block_R(w.V, I, J, R)
        assert missed <= 1e-12 * hmax
        for i, q in enumerate(qs):
            blk = HR[off[q]:off[q + 1]].reshape(ref[i].shape)
            assert np.abs(blk - ref[i]).max() <= TOL * hmax, (I, J, tuple(R[i]))
    g.close()


def test_folded_cell_every_key_against_the_oracle():
    """8-atom cubic Si cell (bricks see several images of one atom): every (I, J) pair's H(R), all R,
    against the oracle's per-image-pair sum, which also confirms that no image pair is missing from
    the keys; includes on-site keys (I, I, R != 0) of an atom and its own images."""
    import torch

    from paper_2603_21835_gb300 import gint as G

    w = inputs.config_workload("si8_g48")
    g = G.Gint(w.system)
    keys, off = g.layout_R()
    V = torch.from_numpy(np.ascontiguousarray(w.V.reshape(-1))).cuda()
    HR = g.vlocal_R(V, G.F16X3).cpu().numpy()
    g.sync()
    o = Oracle(w.system)
    hmax = np.abs(HR).max()
    assert any(k[0] == k[1] and any(k[2:]) for k in keys)
    for I in range(w.system.natoms):
        for J in range(w.system.natoms):
            qs = [q for q, k in enumerate(keys) if k[0] == I and k[1] == J]
            assert qs, (I, J)
            ref, missed = o.vlocal_block_R(w.V, I, J, keys[qs, 2:])
            assert missed <= 1e-12 * hmax, (I, J, missed)
            for i, q in enumerate(qs):
                blk = HR[off[q]:off[q + 1]].reshape(ref[i].shape)
                assert np.abs(blk - ref[i]).max() <= TOL * hmax, (I, J, tuple(keys[q, 2:]))
    g.close()


def test_folded_cell_follows_new_positions():
    """Positions moved within the skin: the folded handle's H(R) (its twin moved with it) against the
    oracle of the moved cell."""
    import dataclasses

    import torch

    from paper_2603_21835_gb300 import gint as G

    w = inputs.config_workload("si8_g48")
    g = G.Gint(w.system, skin=0.5)
    g.layout_R()  # the twin exists before the move
    pos = w.system.pos + np.random.default_rng(8).normal(0.0, 0.08, w.system.pos.shape)
    g.set_positions(torch.from_numpy(np.ascontiguousarray(pos)).cuda())
    keys, off = g.layout_R()
    V = torch.from_numpy(np.ascontiguousarray(w.V.reshape(-1))).cuda()
    HR = g.vlocal_R(V, G.F16X3).cpu().numpy()
    g.sync()
    o = Oracle(dataclasses.replace(w.system, pos=pos))
    hmax = np.abs(HR).max()
    for I, J in [(0, 0), (1, 6), (4, 4)]:
        qs = [q for q, k in enumerate(keys) if k[0] == I and k[1] == J]
        ref, missed = o.vlocal_block_R(w.V, I, J, keys[qs, 2:])
        assert missed <= 1e-12 * hmax
        for i, q in enumerate(qs):
            assert np.abs(HR[off[q]:off[q + 1]].reshape(ref[i].shape) - ref[i]).max() <= TOL * hmax
    g.close()
