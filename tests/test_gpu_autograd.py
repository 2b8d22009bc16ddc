"""Differentiation of E = sum_g w V rho: hand-written backward against gradcheck, central
finite differences (step 1e-4 Bohr) and the oracle's force (paper Sec. 3.3.1, local Pulay force).

Finite differences use the float64 path (its energy is exact to ~1e-14, so the difference
quotient is limited by the h^2 truncation); the mixed-precision forces are compared with the
float64 forces and the oracle at the force tolerance 1e-5 Ha/Bohr."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2603_21835_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch

    from paper_2603_21835_gb300 import autograd as A
    from paper_2603_21835_gb300 import gint as G

    return torch, G, A


def test_gradcheck_small_cell(mods):
    torch, G, A = mods
    w = inputs.si_workload((1, 1, 1), (16, 16, 16), seed=3, disp_sigma=0.08)
    sysm = inputs.System(cell=w.system.cell, pos=w.system.pos[[0, 3, 5]], species=np.zeros(3, np.int32),
                         sp=w.system.sp, grid=w.system.grid)
    g = G.Gint(sysm, skin=0.5)
    rng = np.random.default_rng(0)
    C = rng.normal(size=(g.norb, 4)) / 4
    Db = torch.from_numpy(g.dense_to_blocks(C @ C.T)).cuda()
    V = torch.from_numpy(w.V.reshape(-1)).cuda().requires_grad_(True)
    pos = torch.from_numpy(sysm.pos.copy()).cuda().requires_grad_(True)
    f = lambda V_, pos_: A.grid_energy(g, Db, V_, pos_, G.FP64)
    assert torch.autograd.gradcheck(f, (V, pos), eps=1e-5, atol=1e-7, rtol=1e-5, nondet_tol=1e-12)
    # dE/dD = H against a symmetric directional derivative
    Dr = Db.clone().requires_grad_(True)
    E = A.grid_energy(g, Dr, V.detach(), pos.detach(), G.FP64)
    (gD,) = torch.autograd.grad(E, Dr)
    S = g.dense_to_blocks(np.eye(g.norb) + 0.3 * (lambda M: M + M.T)(rng.normal(size=(g.norb, g.norb))))
    S = torch.from_numpy(S).cuda()
    eps = 1e-4
    Ep = A.grid_energy(g, Db + eps * S, V.detach(), pos.detach(), G.FP64).item()
    Em = A.grid_energy(g, Db - eps * S, V.detach(), pos.detach(), G.FP64).item()
    assert (Ep - Em) / (2 * eps) == pytest.approx(torch.dot(gD, S).item(), rel=1e-9)
    g.close()


@pytest.fixture(scope="module")
def si64d(mods):
    torch, G, A = mods
    w = inputs.config_workload("si64_g96_d")
    g = G.Gint(w.system, skin=0.5)
    Db = torch.from_numpy(g.dense_to_blocks(w.D)).cuda()
    V = torch.from_numpy(w.V.reshape(-1)).cuda()
    return w, g, Db, V


@pytest.mark.parametrize("prec", ["fp64", "f16x3"])
def test_forces_vs_central_differences_and_oracle(mods, si64d, prec):
    """64-atom Si cell, N(0, 0.1) Bohr displacements, 96^3 grid."""
    torch, G, A = mods
    w, g, Db, V = si64d
    p = G.PRECISIONS[prec]
    pos0 = torch.from_numpy(w.system.pos.copy()).cuda()
    pos = pos0.clone().requires_grad_(True)
    E = A.grid_energy(g, Db, V, pos, p)
    (dEdR,) = torch.autograd.grad(E, pos)
    F = -dEdR.cpu().numpy()
    # finite differences of the float64 energy on a sample of coordinates
    atoms = [0, 17, 42, 63]
    h = 1e-4
    for I in atoms:
        for c in range(3):
            Es = []
            for sgn in (1, -1):
                q = pos0.clone()
                q[I, c] += sgn * h
                Es.append(A.grid_energy(g, Db, V, q, G.FP64).item())
            fd = -(Es[0] - Es[1]) / (2 * h)
            assert abs(F[I, c] - fd) <= 1e-5, (prec, I, c, F[I, c], fd)
    g.ensure_positions(pos0)
    # the oracle's local Pulay force on all 64 atoms
    Fo = _oracle_forces(w)
    err = np.abs(F - Fo).max()
    worst = np.argsort(-np.abs(F - Fo).max(1))[:4]
    print(prec, "forces of all 64 atoms vs the oracle:", err, "Ha/Bohr; worst atoms",
          [(int(a), float(np.abs(F - Fo)[a].max())) for a in worst])
    assert err <= (1e-11 * np.abs(Fo).max() if prec == "fp64" else 1e-5)


_FO = {}


def _oracle_forces(w):
    if "F" not in _FO:
        _FO["F"] = Oracle(w.system).force(w.D, w.V)
    return _FO["F"]
