"""Pins for the oracle's density-matrix build and Crank-Nicolson step (oracle/dense.py): properties the
mathematics fixes, checked with routines other than the oracle's own (a generalised symmetric eigen-
solver, explicit loops)."""
import numpy as np
import scipy.linalg

from oracle.dense import crank_nicolson, density_matrix, energy_density_matrix


def _matrices(n=60, seed=0):
    rng = np.random.default_rng(seed)
    Q = rng.normal(size=(n, n))
    S = np.eye(n) + 0.5 * (Q @ Q.T) / n  # symmetric positive definite, like an overlap matrix
    G = rng.normal(size=(n, n))
    H = 0.5 * (G + G.T)
    return S, H


def test_cn_conserves_the_S_norm():
    """The Cayley transform is unitary in the S metric: psi'^dagger S psi' = psi^dagger S psi."""
    S, H = _matrices()
    rng = np.random.default_rng(1)
    psi = rng.normal(size=(60, 7)) + 1j * rng.normal(size=(60, 7))
    out = crank_nicolson(S, H, 0.1, psi)
    g0, g1 = psi.conj().T @ S @ psi, out.conj().T @ S @ out
    assert np.abs(g1 - g0).max() <= 1e-12 * np.abs(g0).max()


def test_cn_on_eigenstates_is_the_cayley_phase():
    """For H c = e S c the step multiplies c by (1 - i dt e / 2) / (1 + i dt e / 2)."""
    S, H = _matrices(seed=2)
    e, C = scipy.linalg.eigh(H, S)
    dt = 0.07
    psi = C[:, :9].astype(np.complex128)
    out = crank_nicolson(S, H, dt, psi)
    ph = (1 - 0.5j * dt * e[:9]) / (1 + 0.5j * dt * e[:9])
    assert np.abs(out - psi * ph[None, :]).max() <= 1e-12


def test_cn_is_time_reversible():
    S, H = _matrices(seed=3)
    rng = np.random.default_rng(4)
    psi = rng.normal(size=(60, 5)) + 1j * rng.normal(size=(60, 5))
    back = crank_nicolson(S, H, -0.2, crank_nicolson(S, H, 0.2, psi))
    assert np.abs(back - psi).max() <= 1e-12 * np.abs(psi).max()


def test_density_matrix_by_explicit_sum_and_trace():
    rng = np.random.default_rng(5)
    n, k = 40, 6
    psi = rng.normal(size=(n, k)) + 1j * rng.normal(size=(n, k))
    f = rng.uniform(0, 2, size=k)
    D = density_matrix(psi, f)
    ref = np.zeros((n, n))
    for s in range(k):
        for i in range(n):
            for j in range(n):
                ref[i, j] += f[s] * (psi[i, s] * np.conj(psi[j, s])).real
    assert np.abs(D - ref).max() <= 1e-13 * np.abs(ref).max()
    # S-orthonormal states: Tr(D S) = sum of the occupations
    S, H = _matrices(n=n, seed=6)
    e, C = scipy.linalg.eigh(H, S)
    D2 = density_matrix(C[:, :k], f)
    assert abs(np.trace(D2 @ S) - f.sum()) <= 1e-12 * f.sum()


def test_edm_of_eigenstates_is_the_textbook_form():
    """For S-orthonormal eigenstates (H c = e S c) and D = C f C^T: E = C f e C^T."""
    S, H = _matrices(seed=7)
    e, C = scipy.linalg.eigh(H, S)
    k = 11
    f = np.random.default_rng(8).uniform(0, 2, size=k)
    D = (C[:, :k] * f) @ C[:, :k].T
    E = energy_density_matrix(S, H, D)
    ref = (C[:, :k] * (f * e[:k])) @ C[:, :k].T
    assert np.abs(E - ref).max() <= 1e-12 * np.abs(ref).max()


def test_edm_identities():
    S, H = _matrices(seed=9)
    rng = np.random.default_rng(10)
    G = rng.normal(size=S.shape)
    D = 0.5 * (G + G.T)
    E = energy_density_matrix(S, H, D)
    assert np.abs(E - E.T).max() == 0.0
    assert abs(np.trace(E @ S) - np.trace(H @ D)) <= 1e-12 * np.abs(H @ D).sum()
    E1 = energy_density_matrix(np.eye(S.shape[0]), H, D)
    assert np.abs(E1 - 0.5 * (H @ D + D @ H)).max() <= 1e-13 * np.abs(H @ D).max()
