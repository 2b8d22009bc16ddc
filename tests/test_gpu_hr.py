"""GPU parity of the local H per lattice vector, H_IJ(R), and its Bloch sum H(k) = sum_R e^{ik.R} H(R)
(paper Sec. 2; the local-potential matrix element of Sec. 3.3.1) against the FP64 oracle on the same
seeded inputs.  Tolerance of the tensor-core F16X3 path: 1e-6 of max |H| (max-norm relative)."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2603_21835_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-6


@pytest.fixture(scope="module")
def si64():
    import torch

    from paper_2603_21835_gb300 import gint as G

    w = inputs.config_workload("si64_g96")
    g = G.Gint(w.system)
    keys, off = g.layout_R()
    V = torch.from_numpy(np.ascontiguousarray(w.V.reshape(-1))).cuda()
    HR_dev = g.vlocal_R(V, G.F16X3)
    H = g.vlocal(V, G.F16X3).cpu().numpy()
    g.sync()
    return dict(w=w, g=g, G=G, keys=keys, off=off, HR_dev=HR_dev, HR=HR_dev.cpu().numpy(), H=H, o=Oracle(w.system),
                torch=torch)


def _block(s, q):
    I, J = s["keys"][q, :2]
    nI, nJ = s["o"]._norb_atom(I), s["o"]._norb_atom(J)
    return s["HR"][s["off"][q]:s["off"][q + 1]].reshape(nI, nJ)


def test_keys_closed_under_transposition(si64):
    s = si64
    keys = s["keys"]
    assert len(keys) > 0 and np.all(np.diff(s["off"]) > 0)
    index = {tuple(k): q for q, k in enumerate(keys)}
    assert [tuple(k) for k in keys] == sorted(index)  # sorted by (I, J, n1, n2, n3)
    hmax = np.abs(s["HR"]).max()
    for q, k in enumerate(keys):
        t = index[(k[1], k[0], -k[2], -k[3], -k[4])]
        if k[0] != k[1]:
            assert np.array_equal(_block(s, t), _block(s, q).T)  # one sum, written twice
        else:  # on-site (R = 0): symmetric to the split products' rounding
            assert t == q and np.abs(_block(s, q) - _block(s, q).T).max() <= TOL * hmax


def test_sum_over_R_is_the_gamma_block(si64):
    s = si64
    g, keys = s["g"], s["keys"]
    acc = np.zeros_like(s["H"])
    for q, k in enumerate(keys):
        p = g.block_index(int(k[0]), int(k[1]))
        assert p >= 0
        acc[g.pair_off[p]:g.pair_off[p + 1]] += s["HR"][s["off"][q]:s["off"][q + 1]]
    assert np.abs(acc - s["H"]).max() <= 1e-9 * np.abs(s["H"]).max()


def _pair_keys(s, I, J):
    return [q for q, k in enumerate(s["keys"]) if k[0] == I and k[1] == J]


def test_sampled_blocks_match_the_oracle(si64):
    """Every R of a few atom pairs (on-site, nearest and farther neighbours) against the oracle, which
    also confirms that no overlapping image pair is missing from the key list."""
    s = si64
    hmax = np.abs(s["HR"]).max()
    pairs = [(0, 0), (0, 1), (5, 40), (63, 2)]
    for I, J in pairs:
        qs = _pair_keys(s, I, J)
        assert qs, (I, J)
        R = s["keys"][qs, 2:]
        ref, missed = s["o"].vlocal_block_R(s["w"].V, I, J, R)
        assert missed <= 1e-12 * hmax, (I, J, missed)
        for i, q in enumerate(qs):
            assert np.abs(_block(s, q) - ref[i]).max() <= TOL * hmax, (I, J, tuple(R[i]))


def test_bloch_sum(si64):
    s = si64
    g, torch = s["g"], s["torch"]
    Hk0 = g.bloch(s["HR_dev"], [0.0, 0.0, 0.0]).cpu().numpy()
    assert np.all(Hk0.imag == 0.0)
    assert np.abs(Hk0.real - s["H"]).max() <= 1e-9 * np.abs(s["H"]).max()
    kf = np.array([0.25, 0.1, -0.3])
    Hk = g.bloch(s["HR_dev"], kf).cpu().numpy()
    g.sync()
    hmax = np.abs(s["HR"]).max()
    # Hermitian: H_JI(k) = H_IJ(k)^dagger
    for I, J in [(0, 1), (5, 40), (63, 2)]:
        p, t = g.block_index(I, J), g.block_index(J, I)
        nI, nJ = s["o"]._norb_atom(I), s["o"]._norb_atom(J)
        A = Hk[g.pair_off[p]:g.pair_off[p + 1]].reshape(nI, nJ)
        B = Hk[g.pair_off[t]:g.pair_off[t + 1]].reshape(nJ, nI)
        assert np.abs(B - A.conj().T).max() <= 1e-12 * hmax
    # against the oracle's H(R) summed with the phases
    for I, J in [(0, 1), (63, 2)]:
        qs = _pair_keys(s, I, J)
        R = s["keys"][qs, 2:]
        ref, _ = s["o"].vlocal_block_R(s["w"].V, I, J, R)
        ph = np.exp(2j * np.pi * (R @ kf))
        refk = np.tensordot(ph, ref, axes=1)
        p = g.block_index(I, J)
        A = Hk[g.pair_off[p]:g.pair_off[p + 1]].reshape(refk.shape)
        assert np.abs(A - refk).max() <= len(qs) * TOL * hmax


def test_several_k_points_in_one_call(si64):
    """Nine k points (two launches of up to eight) equal nine single-k calls."""
    s = si64
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


def test_folded_cell_is_unsupported():
    """8-atom Si cell: a brick sees two images of an atom, so its tiles mix R."""
    from paper_2603_21835_gb300 import gint as G

    w = inputs.config_workload("si8_g48")
    g = G.Gint(w.system)
    with pytest.raises(G.GintError, match="-8|unsupported|UNSUPPORTED"):
        g.layout_R()
    g.close()
