"""Dense-matrix steps of real-time propagation that consume the grid matrices, in plain float64 /
complex128 numpy and LAPACK (scipy): the density-matrix build from coefficients and occupations, and
one Crank-Nicolson step of the coefficients.

TEST INFRASTRUCTURE ONLY: the test-suite and the CPU-baseline leg of the benchmark use this module;
the product path never imports it, and it imports nothing from the CUDA library or its binding.

Paper references: the density matrix rho_{mu nu} = sum_n f_n c_{mu n} c*_{nu n} (Sec. 2, at the Gamma
point its real part enters the grid density); the Crank-Nicolson propagator
(S + i dt/2 H) C(t + dt) = (S - i dt/2 H) C(t) solved by an LU factorisation (Sec. 2, time
propagation of the coefficients with the overlap matrix S); the energy-density matrix
E = (S^{-1} H rho + rho H S^{-1}) / 2 that the overlap part of the forces needs.
"""
import numpy as np
import scipy.linalg


def density_matrix(psi: np.ndarray, f: np.ndarray) -> np.ndarray:
    """D = Re(psi diag(f) psi^dagger): psi [n, nocc] complex (columns are states), f [nocc]."""
    psi = np.asarray(psi, dtype=np.complex128)
    return np.real((psi * np.asarray(f, dtype=np.float64)[None, :]) @ psi.conj().T)


def crank_nicolson(S: np.ndarray, H: np.ndarray, dt: float, psi: np.ndarray) -> np.ndarray:
    """psi(t + dt) = (S + i dt/2 H)^{-1} (S - i dt/2 H) psi(t) by LU with partial pivoting (LAPACK
    zgetrf / zgetrs); S, H [n, n] real symmetric, psi [n, nocc] complex."""
    S = np.asarray(S, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    A = S + 0.5j * dt * H
    B = (S - 0.5j * dt * H) @ np.asarray(psi, dtype=np.complex128)
    return scipy.linalg.lu_solve(scipy.linalg.lu_factor(A), B)


def energy_density_matrix(S: np.ndarray, H: np.ndarray, D: np.ndarray) -> np.ndarray:
    """E = (S^{-1} H D + D H S^{-1}) / 2 for real symmetric S (positive definite), H and D: with
    X = S^{-1} H D (a Cholesky solve, LAPACK dpotrf / dpotrs) the second term is X^T."""
    X = scipy.linalg.cho_solve(scipy.linalg.cho_factor(np.asarray(S, dtype=np.float64)),
                               np.asarray(H, dtype=np.float64) @ np.asarray(D, dtype=np.float64))
    return 0.5 * (X + X.T)
