"""GPU parity of the density-matrix build, the Crank-Nicolson step (paper Sec. 2) and the energy-
density matrix (the library's own float64 GEMM and blocked L D L^T kernels) against the LAPACK oracle
(oracle/dense.py, LU with partial pivoting and Cholesky), all in float64: 1e-12 of the largest
entry; the tensor-core density-matrix build (float16 three-term split) within 1e-6 of
max_i sum_s |f_s| |psi_is|^2; and the loop rho -> H -> psi -> rho closed on the 8-atom Si cell with
the grid library's own passes."""
import numpy as np
import pytest

from oracle.dense import crank_nicolson, density_matrix, energy_density_matrix
from oracle.oracle import Oracle
from paper_2603_21835_gb300 import inputs

pytestmark = pytest.mark.gpu


def _matrices(n, seed):
    rng = np.random.default_rng(seed)
    Q = rng.normal(size=(n, n))
    S = np.eye(n) + 0.5 * (Q @ Q.T) / n
    G = rng.normal(size=(n, n))
    return S, 0.5 * (G + G.T)


@pytest.mark.parametrize("n,k", [(832, 64), (130, 3), (1601, 33)])
def test_step_and_density_matrix_match_the_oracle(n, k):
    """Sizes on and off the 64-wide blocks of the factorisation and of the GEMM tiles."""
    import torch

    from paper_2603_21835_gb300 import gint as G

    S, H = _matrices(n, 0)
    rng = np.random.default_rng(1)
    psi = rng.normal(size=(n, k)) + 1j * rng.normal(size=(n, k))
    f = rng.uniform(0, 2, size=k)
    cn = G.CrankNicolson(n, k)
    Sd, Hd = torch.from_numpy(S).cuda(), torch.from_numpy(H).cuda()
    pd = torch.from_numpy(np.ascontiguousarray(psi.T)).cuda()  # rows are states
    out = cn.step(Sd, Hd, 0.05, pd).cpu().numpy().T
    D = cn.density_matrix(pd, torch.from_numpy(f).cuda()).cpu().numpy()
    assert cn.info() == 0
    ref = crank_nicolson(S, H, 0.05, psi)
    assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()
    Dref = density_matrix(psi, f)
    assert np.abs(D - Dref).max() <= 1e-12 * np.abs(Dref).max()
    assert np.array_equal(D, D.T)  # lower triangle computed and mirrored
    cn.close()


@pytest.mark.parametrize("n", [832, 130, 1601])
def test_energy_density_matrix_matches_the_oracle(n):
    import torch

    from paper_2603_21835_gb300 import gint as G

    S, H = _matrices(n, 2)
    G_ = np.random.default_rng(3).normal(size=(n, n))
    D = 0.5 * (G_ + G_.T)
    cn = G.CrankNicolson(n, 8)
    E = cn.energy_density_matrix(*(torch.from_numpy(x).cuda() for x in (S, H, D))).cpu().numpy()
    assert cn.info() == 0
    ref = energy_density_matrix(S, H, D)
    assert np.abs(E - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(E - E.T).max() == 0.0
    cn.close()


def test_energy_density_matrix_reports_a_non_positive_pivot():
    """S with a negative eigenvalue in its 70th leading block: the factorisation's info names the
    first non-positive pivot (the 70th, in the second 64-wide block)."""
    import torch

    from paper_2603_21835_gb300 import gint as G

    n = 100
    S = np.eye(n)
    S[69, 69] = -1.0
    H, D = np.eye(n), np.eye(n)
    cn = G.CrankNicolson(n, 4)
    cn.energy_density_matrix(*(torch.from_numpy(x).cuda() for x in (S, H, D)))
    assert cn.info() == 70
    # the next call starts from a clean info word
    S[69, 69] = 2.0
    cn.energy_density_matrix(*(torch.from_numpy(x).cuda() for x in (S, H, D)))
    assert cn.info() == 0
    cn.close()


def test_loop_rho_H_psi_rho_on_the_grid():
    """S = H_grid(V = 1), H = H_grid(V), psi from the workload's coefficients: one step, the new
    density matrix, and its density on the grid, all on the GPU (float64), against the oracle chain."""
    import torch

    from paper_2603_21835_gb300 import gint as G

    w = inputs.config_workload("si8_g48")
    g = G.Gint(w.system)
    o = Oracle(w.system)
    V = torch.from_numpy(np.ascontiguousarray(w.V.reshape(-1))).cuda()
    one = torch.ones_like(V)
    S = g.blocks_to_dense(g.vlocal(one, G.FP64).cpu().numpy())
    H = g.blocks_to_dense(g.vlocal(V, G.FP64).cpu().numpy())
    n = S.shape[0]
    C = np.asarray(w.C)[:, :16]
    f = np.full(C.shape[1], 2.0)
    cn = G.CrankNicolson(n, C.shape[1])
    pd = torch.from_numpy(np.ascontiguousarray(C.T.astype(np.complex128))).cuda()
    out = cn.step(torch.from_numpy(S).cuda(), torch.from_numpy(H).cuda(), 0.1, pd)
    D = cn.density_matrix(out, torch.from_numpy(f).cuda()).cpu().numpy()
    rho = g.rho(torch.from_numpy(g.dense_to_blocks(D)).cuda(), G.FP64).cpu().numpy().reshape(-1)
    g.sync()
    So, Ho = o.vlocal(np.ones(o.ngrid)), o.vlocal(w.V)
    Dref = density_matrix(crank_nicolson(So, Ho, 0.1, C.astype(np.complex128)), f)
    rref = o.rho(Dref).reshape(-1)
    # both sides agree on S and H to ~1e-12; the solve amplifies that by the condition number
    cond = np.linalg.cond(So + 0.05j * Ho)
    assert np.abs(D - Dref).max() <= 1e-8 * np.abs(Dref).max(), cond
    assert np.abs(rho - rref).max() <= 1e-8 * np.abs(rref).max(), cond
    cn.close()
    g.close()


@pytest.mark.parametrize("n,nocc,signed", [(832, 64, False), (700, 37, True), (130, 3, False), (6656, 1024, False)])
def test_tensor_core_density_matrix(n, nocc, signed):
    """Ragged n (tiles of 128) and K = 2 nocc (chunks of 64), fewer chunks than accumulators (nocc 3),
    occupations of both signs, and the 512-atom size (6656 orbitals, 1024 states) on sampled rows."""
    import torch

    from paper_2603_21835_gb300 import gint as G

    rng = np.random.default_rng(n + nocc)
    psi = (rng.normal(size=(n, nocc)) + 1j * rng.normal(size=(n, nocc))) / 32
    f = rng.uniform(-1, 2, size=nocc) if signed else rng.uniform(0, 2, size=nocc)
    cn = G.CrankNicolson(n, nocc)
    pd = torch.from_numpy(np.ascontiguousarray(psi.T)).cuda()
    D = cn.density_matrix(pd, torch.from_numpy(f).cuda(), precision="f16x3").cpu().numpy()
    assert cn.info() == 0
    cn.close()
    assert np.array_equal(D, D.T)
    bound = (np.abs(psi) ** 2 @ np.abs(f)).max()
    idx = np.arange(n) if n <= 1024 else np.unique(np.r_[rng.choice(n, 300, replace=False), 0, n - 1])
    ref = density_matrix(psi[idx], f)
    err = np.abs(D[np.ix_(idx, idx)] - ref).max()
    print(f"n={n} nocc={nocc}: max error {err / bound:.3g} of max_i sum_s |f_s| |psi_is|^2")
    assert err <= 1e-6 * bound, (err, bound)
    assert err > 0.0  # the float16 path ran, not a float64 one


def test_tensor_core_density_matrix_of_zero_states_is_zero():
    import torch

    from paper_2603_21835_gb300 import gint as G

    cn = G.CrankNicolson(200, 5)
    D = cn.density_matrix(torch.zeros((5, 200), dtype=torch.complex128, device="cuda"),
                          torch.ones(5, dtype=torch.float64, device="cuda"), precision="f16x3")
    assert cn.info() == 0
    assert torch.count_nonzero(D).item() == 0
    cn.close()
