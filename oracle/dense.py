"""Small dense symmetric tools (oracle).

* ``jacobi_eigh``       cyclic Jacobi eigensolver for a real symmetric matrix.
* ``generalized_eigh``  A v = lam S v with S SPD: Cholesky S = C C^T, then Jacobi on
                         C^{-1} A C^{-T}; eigenvalues ascending.  This is the p x p problem
                         of the Rayleigh-Ritz post-processing (Sec. 4.3).
* ``scf``               a dense linear-mixing self-consistent field loop on tiny meshes
                         (Sec. 5 describes SCF with density mixing as the comparison
                         method).  Used only to pin the nonlinear fixed point that PCAL
                         must reach, by an algorithm that shares nothing with PCAL's update.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def jacobi_eigh(A: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """Eigen-decomposition of symmetric A by cyclic Jacobi rotations.

    Each rotation in the (i, j) plane zeroes a_ij: with theta = (a_jj - a_ii) / (2 a_ij)
    the tangent t = sign(theta) / (|theta| + sqrt(theta^2 + 1)) solves t^2 + 2 theta t = 1.
    Returns (w ascending, V) with A V = V diag(w).
    """
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    V = np.eye(n)
    scale = max(np.linalg.norm(A), 1e-300)
    for _ in range(max_sweeps):
        off = np.sqrt(max(np.sum(A * A) - np.sum(np.diag(A) ** 2), 0.0))
        if off <= tol * scale:
            break
        for i in range(n - 1):
            for j in range(i + 1, n):
                aij = A[i, j]
                if aij == 0.0:
                    continue
                theta = (A[j, j] - A[i, i]) / (2.0 * aij)
                t = (1.0 if theta >= 0 else -1.0) / (abs(theta) + np.hypot(theta, 1.0))
                c = 1.0 / np.sqrt(t * t + 1.0)
                s = t * c
                ci, cj = A[:, i].copy(), A[:, j].copy()
                A[:, i], A[:, j] = c * ci - s * cj, s * ci + c * cj
                ri, rj = A[i, :].copy(), A[j, :].copy()
                A[i, :], A[j, :] = c * ri - s * rj, s * ri + c * rj
                vi, vj = V[:, i].copy(), V[:, j].copy()
                V[:, i], V[:, j] = c * vi - s * vj, s * vi + c * vj
    w = np.diag(A).copy()
    order = np.argsort(w, kind="stable")
    return w[order], V[:, order]


def generalized_eigh(A: np.ndarray, S: np.ndarray):
    """Solve A v = lam S v (A symmetric, S SPD); returns (lam ascending, V) with V^T S V = I."""
    C = np.linalg.cholesky(S)                              # S = C C^T
    Ci = np.linalg.inv(C)
    At = Ci @ A @ Ci.T
    At = 0.5 * (At + At.T)
    w, W = jacobi_eigh(At)
    return w, Ci.T @ W


def scf(problem, X0: np.ndarray, alpha: float = 0.5, tol: float = 1e-12, max_iter: int = 2000):
    """Dense SCF with linear density mixing rho <- alpha rho_new + (1 - alpha) rho.

    Each step assembles H(rho) and takes the p lowest generalized eigenvectors of the dense
    pencil (H, B) (LAPACK through scipy: the n x n problem is too large for plain Jacobi).  Stops when the change of the density (quadrature-weighted L1) is below tol.
    Returns (X, E_total, eigenvalues, iterations).
    """
    p = X0.shape[1]
    Bd = problem.Bf.toarray()
    rho = problem.density(X0)
    X = X0
    w = None
    for it in range(1, max_iter + 1):
        pot = problem.potentials(rho)
        Hd = problem.hamiltonian(pot).toarray()
        w, X = sla.eigh(Hd, Bd, subset_by_index=[0, p - 1])
        rho_new = problem.density(X)
        change = float(np.sum(problem.wq2 * np.abs(rho_new - rho)))
        rho = alpha * rho_new + (1.0 - alpha) * rho
        if change < tol:
            break
    E = problem.energy(X)["total"]
    return X, E, w, it
