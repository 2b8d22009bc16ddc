"""GPU parity: the CUDA passes against the FP64 oracle on the same seeded inputs.

Error metric (max-norm relative): err(X) = max|X - X_ref| / max|X_ref| for rho and H; forces
in absolute Ha/Bohr.  Tolerances: FP64 path 1e-12 (relative; forces 1e-11 of max|F|),
tensor-core F16x3 path 1e-6 (rho, H) and 1e-5 Ha/Bohr (forces), float32 SIMT 1e-5.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2603_21835_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "f16x3": 1e-6}
FTOL_ABS = {"fp64": None, "fp32": 1e-5, "f16x3": 1e-5}


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    from paper_2603_21835_gb300 import gint  # noqa: F401  (fails loudly without the library)

    return torch


def _run(G, g, D_blocks, V, prec, torch):
    Dd = torch.from_numpy(D_blocks).cuda()
    Vd = torch.from_numpy(np.ascontiguousarray(V.reshape(-1))).cuda()
    rho = g.rho(Dd, prec).cpu().numpy()
    H = g.vlocal(Vd, prec).cpu().numpy()
    rho2 = torch.empty(g.grid, dtype=torch.float64, device="cuda")
    F = g.force(Dd, Vd, prec, rho_out=rho2).cpu().numpy()
    torch.cuda.synchronize()
    return rho, H, F, rho2.cpu().numpy()


class Case:
    def __init__(self, w, torch):
        from paper_2603_21835_gb300 import gint as G

        self.w = w
        self.o = Oracle(w.system)
        self.g = G.Gint(w.system)
        self.G = G
        self.rho = self.o.rho(w.D)
        self.H = self.o.vlocal(w.V)
        self.F = self.o.force(w.D, w.V)
        self.Db = self.g.dense_to_blocks(w.D)


@pytest.fixture(scope="module")
def si8(torch_cuda):
    return Case(inputs.config_workload("si8_g48"), torch_cuda)


def test_tc_mma_selftest(torch_cuda):
    """One tcgen05 kind::f16 MMA per operand layout on exact integer data."""
    from paper_2603_21835_gb300 import gint as G

    for n in (16, 32, 112, 208, 256):
        assert G.tc_selftest(n) == 0.0


@pytest.mark.parametrize("prec", ["fp64", "fp32", "f16x3"])
def test_si8_parity(si8, torch_cuda, prec):
    c = si8
    p = c.G.PRECISIONS[prec]
    rho, H, F, rho2 = _run(c.G, c.g, c.Db, c.w.V, p, torch_cuda)
    c.g.sync()
    Hd = c.g.blocks_to_dense(H)
    print(prec, "rho", _rel(rho, c.rho), "H", _rel(Hd, c.H), "F", np.abs(F - c.F).max())
    assert _rel(rho, c.rho) <= TOL[prec]
    assert _rel(rho2, c.rho) <= TOL[prec]
    assert _rel(Hd, c.H) <= TOL[prec]
    if prec == "fp64":
        assert np.abs(F - c.F).max() <= 1e-11 * np.abs(c.F).max()
    else:
        assert np.abs(F - c.F).max() <= FTOL_ABS[prec]


def test_si8_work_count(si8):
    st = si8.g.stats()
    W, _ = si8.o.count_pairs()
    assert st["W"] == W
    assert st["W_exec"] >= W


def test_si8_identities_on_device(si8, torch_cuda):
    """sum_g w rho = Tr(DS) and sum_g w V rho = Tr(DH), all reductions on the device in FP64."""
    torch = torch_cuda
    c = si8
    Dd = torch.from_numpy(c.Db).cuda()
    V = torch.from_numpy(c.w.V.reshape(-1)).cuda()
    one = torch.ones_like(V)
    rho = c.g.rho(Dd)
    S = c.g.vlocal(one)
    H = c.g.vlocal(V)
    ne = c.g.grid_dot(None, rho).item()
    trDS = c.g.block_dot(Dd, S).item()
    E = c.g.grid_dot(V, rho).item()
    trDH = c.g.block_dot(Dd, H).item()
    assert ne == pytest.approx(trDS, rel=1e-12)
    assert E == pytest.approx(trDH, rel=1e-12)
    Hn = c.g.blocks_to_dense(H.cpu().numpy())
    assert np.abs(Hn - Hn.T).max() <= 1e-14 * np.abs(Hn).max()


def _small_case(torch, system, seed=3, nb=6):
    from paper_2603_21835_gb300 import gint as G

    rng = np.random.default_rng(seed)
    o = Oracle(system)
    C = rng.normal(size=(o.norb, nb)) / 4
    D = C @ C.T
    V = inputs.draw_V(rng, system.cell, system.grid).reshape(-1)
    g = G.Gint(system)
    rho_o, H_o, F_o = o.rho(D).reshape(-1), o.vlocal(V), o.force(D, V)
    for prec, tol in (("fp64", 1e-12), ("f16x3", 1e-6)):
        rho, H, F, rho2 = _run(G, g, g.dense_to_blocks(D), V, G.PRECISIONS[prec], torch)
        g.sync()
        assert _rel(rho.reshape(-1), rho_o) <= tol, prec
        assert _rel(rho2.reshape(-1), rho_o) <= tol, prec
        assert _rel(g.blocks_to_dense(H), H_o) <= tol, prec
        if prec == "fp64":
            assert np.abs(F - F_o).max() <= 1e-11 * np.abs(F_o).max()
        else:
            assert np.abs(F - F_o).max() <= 1e-5
    return g


def test_ragged_grid(torch_cuda):
    """Grid not divisible by the 4x4x8 brick: partial bricks on every axis."""
    w = inputs.si_workload((1, 1, 1), (21, 18, 27), seed=2, disp_sigma=0.07)
    _small_case(torch_cuda, w.system)


def test_triclinic_cell_with_folded_images(torch_cuda):
    """fcc primitive cell smaller than the orbital diameter: many images of one atom fold."""
    sp = inputs.si_species()
    a = inputs.SI_A
    cell = np.array([[0, a / 2, a / 2], [a / 2, 0, a / 2], [a / 2, a / 2, 0]])
    pos = np.array([[0.0, 0.0, 0.0], [a / 4, a / 4, a / 4]]) + 0.031
    sysm = inputs.System(cell=cell, pos=pos, species=np.zeros(2, np.int32), sp=[sp], grid=(20, 20, 24))
    _small_case(torch_cuda, sysm)


def test_vacuum_and_two_species(torch_cuda):
    """Water molecules in a box: empty bricks, two species with different orbital counts."""
    w = inputs.h2o_workload(2, seed=5, box=16.0, grid=(40, 40, 40))
    _small_case(torch_cuda, w.system)


@pytest.fixture(scope="module")
def si64(torch_cuda):
    w = inputs.config_workload("si64_g96")
    o = Oracle(w.system)
    from paper_2603_21835_gb300 import gint as G

    g = G.Gint(w.system)
    rng = np.random.default_rng(123)
    idx = rng.choice(o.ngrid, 3000, replace=False)
    return dict(w=w, o=o, g=g, G=G, idx=idx, rho=o.rho(w.D, idx), Db=g.dense_to_blocks(w.D))


@pytest.mark.parametrize("prec", ["fp64", "f16x3"])
def test_si64_sampled_parity(si64, torch_cuda, prec):
    torch = torch_cuda
    s = si64
    g, o, w = s["g"], s["o"], s["w"]
    p = s["G"].PRECISIONS[prec]
    Dd = torch.from_numpy(s["Db"]).cuda()
    Vd = torch.from_numpy(w.V.reshape(-1)).cuda()
    rho = g.rho(Dd, p).cpu().numpy().reshape(-1)
    assert _rel(rho[s["idx"]], s["rho"]) <= TOL[prec]
    H = g.vlocal(Vd, p).cpu().numpy()
    g.sync()
    # blocks compared against the max-norm of H (the error metric), sampled pairs
    hmax = np.abs(H).max()
    for (I, J) in [(0, 0), (0, 5), (3, 17), (63, 2), (40, 41), (7, 7)]:
        k = g.block_index(I, J)
        assert k >= 0
        ref = o.vlocal_block(w.V, I, J)
        blk = H[g.pair_off[k]:g.pair_off[k + 1]].reshape(ref.shape)
        assert np.abs(blk - ref).max() <= TOL[prec] * hmax


def test_si64_float64_cross_brick_reduction(si64, torch_cuda):
    """The strict reduction mode (every float32 tile value added in float64) against the default
    double-float sums: the same tiles in the same order, so the two agree far below the tiles'
    own rounding (1e-10 of max|H|; both sums' errors are below 1e-12 here); H(R) as well; and
    against the oracle at the F16x3 tolerance.  The mode is restored afterwards."""
    torch = torch_cuda
    s = si64
    g, o, w, G = s["g"], s["o"], s["w"], s["G"]
    Vd = torch.from_numpy(w.V.reshape(-1)).cuda()
    H_df = g.vlocal(Vd, G.F16X3).cpu().numpy()
    HR_df = g.vlocal_R(Vd, G.F16X3).cpu().numpy()
    g.set_reduction("fp64")
    try:
        H_64 = g.vlocal(Vd, G.F16X3).cpu().numpy()
        HR_64 = g.vlocal_R(Vd, G.F16X3).cpu().numpy()
        g.sync()
    finally:
        g.set_reduction("double-float")
    hmax = np.abs(H_64).max()
    assert np.abs(H_64 - H_df).max() <= 1e-10 * hmax
    assert np.abs(HR_64 - HR_df).max() <= 1e-10 * hmax
    for (I, J) in [(0, 0), (3, 17), (63, 2)]:
        k = g.block_index(I, J)
        ref = o.vlocal_block(w.V, I, J)
        assert np.abs(H_64[g.pair_off[k]:g.pair_off[k + 1]].reshape(ref.shape) - ref).max() <= TOL["f16x3"] * hmax
    with pytest.raises(G.GintError):
        G._check(G._lib.gint_set_reduction(g._h, 7), "gint_set_reduction")


@pytest.fixture(scope="module")
def si512(torch_cuda):
    """512-atom Si (4x4x4 supercell, N(0,0.05) displacements), 192^3 grid, D from C 6656x1024 / 32.
    The oracle runs on the grid sub-volume [0,96)^3 (one eighth of the cell): the density at every
    point of it, and the local H with V zeroed outside it (every block of the pair set)."""
    from paper_2603_21835_gb300 import gint as G

    w = inputs.config_workload("si512_g192", dense_D=True)
    o = Oracle(w.system)
    g = G.Gint(w.system)
    n = np.array(w.system.grid)
    box = np.zeros(tuple(n), bool)
    box[:n[0] // 2, :n[1] // 2, :n[2] // 2] = True
    idx = np.flatnonzero(box.reshape(-1))
    Vbox = np.where(box, w.V, 0.0).reshape(-1)
    return dict(w=w, g=g, G=G, idx=idx, Vbox=Vbox, rho=o.rho(w.D, idx), H=o.vlocal(Vbox, idx),
                Db=g.blocks_from_coefficients(w.C))


@pytest.mark.parametrize("prec", ["fp64", "f16x3"])
def test_si512_subvolume_parity(si512, torch_cuda, prec):
    """Every point of the [0,96)^3 sub-volume (884,736 points) and every H block."""
    torch = torch_cuda
    s = si512
    g = s["g"]
    p = s["G"].PRECISIONS[prec]
    Dd = torch.from_numpy(s["Db"]).cuda()
    Vd = torch.from_numpy(s["Vbox"]).cuda()
    rho = g.rho(Dd, p).cpu().numpy().reshape(-1)
    H = g.blocks_to_dense(g.vlocal(Vd, p).cpu().numpy())
    g.sync()
    er, eh = _rel(rho[s["idx"]], s["rho"]), _rel(H, s["H"])
    print(prec, "rho (884,736 points)", er, "H (all blocks)", eh)
    assert er <= TOL[prec] and eh <= TOL[prec]


@pytest.mark.parametrize("n", [16, 24, 48, 96])
def test_mixed_forces_on_coarse_and_fine_grids(torch_cuda, n):
    """The 8-atom cell (N(0,0.05) displacements) on grids of 16^3 to 96^3: the mixed-precision forces
    within 1e-5 Ha/Bohr of the oracle (absolute), rho and H within 1e-6 (max-norm relative)."""
    from paper_2603_21835_gb300 import gint as G

    w = inputs.si_workload((1, 1, 1), (n, n, n), seed=0, disp_sigma=0.05)
    o = Oracle(w.system)
    g = G.Gint(w.system)
    rho, H, F, rho2 = _run(G, g, g.dense_to_blocks(w.D), w.V, G.F16X3, torch_cuda)
    g.sync()
    Fo = o.force(w.D, w.V)
    ef = np.abs(F - Fo).max()
    er, eh = _rel(rho, o.rho(w.D)), _rel(g.blocks_to_dense(H), o.vlocal(w.V))
    print(f"{n}^3 f16x3: F {ef:.3e} Ha/Bohr (max|F| {np.abs(Fo).max():.2f}), rho {er:.2e}, H {eh:.2e}")
    assert ef <= 1e-5 and er <= 1e-6 and eh <= 1e-6 and _rel(rho2, o.rho(w.D)) <= 1e-6
    g.close()


def test_water_cluster_with_eight_column_atoms(torch_cuda):
    """24 water molecules in a 20 Bohr box, 96^3: O atoms take 16 padded columns, H atoms 8, so
    some bricks end on an 8-column atom (six bricks here have padded width 256 with an H atom at
    columns 248-255, the layout whose force epilogue must read exactly 8 columns)."""
    torch = torch_cuda
    from paper_2603_21835_gb300 import gint as G

    w = inputs.h2o_workload(24, seed=3, box=20.0, grid=(96, 96, 96))
    o = Oracle(w.system)
    g = G.Gint(w.system)
    Db = g.dense_to_blocks(w.D)
    ref_rho, ref_H, ref_F = o.rho(w.D), o.vlocal(w.V), o.force(w.D, w.V)
    for prec in ("fp64", "f16x3"):
        rho, H, F, rho2 = _run(G, g, Db, w.V, G.PRECISIONS[prec], torch)
        g.sync()
        assert _rel(rho, ref_rho) <= TOL[prec], prec
        assert _rel(rho2, ref_rho) <= TOL[prec], prec
        assert _rel(g.blocks_to_dense(H), ref_H) <= TOL[prec], prec
        ftol = FTOL_ABS[prec] if FTOL_ABS[prec] is not None else 1e-11 * np.abs(ref_F).max()
        assert np.abs(F - ref_F).max() <= ftol, prec
    g.close()


@pytest.mark.parametrize("sigma", [1e-6, 0.08])
def test_moved_positions_match_a_fresh_handle(torch_cuda, sigma):
    """gint_set_positions within the skin: a move so small that every brick keeps its atoms (only the
    plan records are rebuilt; a stale record would be off by about the move, 1e-6, against 1e-13
    allowed) and one that changes bricks' atom sets (layouts rebuilt; the pair set kept from
    creation can hold more blocks than a fresh handle's, which can change max|D| and so the float16
    scales: compared at the mixed-precision tolerance).  Either way rho, H and the forces also match
    the oracle at the new positions."""
    import dataclasses

    import torch

    from paper_2603_21835_gb300 import gint as G

    w = inputs.config_workload("si8_g48")
    pos = w.system.pos + np.random.default_rng(11).normal(0.0, sigma, w.system.pos.shape)
    moved = dataclasses.replace(w.system, pos=pos)
    g = G.Gint(w.system, skin=0.5)
    g.set_positions(torch.from_numpy(np.ascontiguousarray(pos)).cuda())
    f = G.Gint(moved, skin=0.5)
    out = []
    for h in (g, f):
        rho, H, F, _ = _run(G, h, h.dense_to_blocks(w.D), w.V, G.F16X3, torch)
        h.sync()
        out.append((rho, h.blocks_to_dense(H), F))
        h.close()
    (rg, Hg, Fg), (rf, Hf, Ff) = out
    same, fsame = (1e-13, 1e-12) if sigma < 1e-3 else (TOL["f16x3"], FTOL_ABS["f16x3"])
    assert _rel(rg, rf) <= same and _rel(Hg, Hf) <= same and np.abs(Fg - Ff).max() <= fsame
    o = Oracle(moved)
    assert _rel(rg, o.rho(w.D).reshape(rg.shape)) <= TOL["f16x3"]
    assert _rel(Hg, o.vlocal(w.V)) <= TOL["f16x3"]
    assert np.abs(Fg - o.force(w.D, w.V)).max() <= FTOL_ABS["f16x3"]
