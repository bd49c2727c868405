"""Hartree potential by the FEM Poisson equation (oracle).

Sec. 2.2: V_Har solves -lap V = 4 pi rho; with V_Har = U^T N the discrete system is
L U = 4 pi (int rho phi_i)_i.  The paper solves it by algebraic multigrid; here the
interior system is solved by a sparse direct factorization (exact up to rounding) on
small meshes, and by Jacobi-preconditioned CG to a 1e-13 relative residual, warm-started
from the previous solution, above DIRECT_MAX_NODES nodes.

Boundary values on the box (the paper is silent on them): the multipole expansion of
rho about the centre c of the node bounding box, up to l = lmax <= 2 (lmax = -1 gives
homogeneous Dirichlet data, for which rho -> V_Har is a symmetric linear map).  With y = x_q - c
    Q    = sum_q w_q rho_q
    d    = sum_q w_q rho_q y
    Q_ij = sum_q w_q rho_q (3 y_i y_j - |y|^2 delta_ij)
    V_B(r) = Q/|r| + d.r/|r|^3 + (1/2) sum_ij Q_ij r_i r_j / |r|^5,   r = x - c.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import fem


DIRECT_MAX_NODES = 40_000


class Hartree:
    def __init__(self, xyz, tet10, dirichlet, L_full, vol, xq, lmax: int = 2, solver: str = "auto"):
        self.xyz, self.tet10, self.vol, self.lmax = xyz, tet10, vol, int(lmax)
        self.n = xyz.shape[0]
        self.center = 0.5 * (xyz.min(axis=0) + xyz.max(axis=0))
        self.I = np.nonzero(dirichlet == 0)[0]
        self.Bd = np.nonzero(dirichlet != 0)[0]
        Lr = L_full[self.I]
        self.L_IB = Lr[:, self.Bd].tocsr()
        L_II = Lr[:, self.I].tocsr()
        if solver == "auto":
            solver = "direct" if self.n <= DIRECT_MAX_NODES else "cg"
        self.solver = solver
        if solver == "direct":
            self.solve_II = spla.factorized(L_II.tocsc())
        else:
            self._L_II = L_II
            self._M = spla.LinearOperator(L_II.shape, matvec=lambda v, d=1.0 / L_II.diagonal(): d * v)
            self._x = np.zeros(len(self.I))
            self.solve_II = self._cg
        self.yq = (xq - self.center).reshape(-1, 3)        # (T*4, 3)
        self.wq = np.repeat(vol / 4.0, 4)

    def moments(self, rho_q):
        """(Q, d (3,), Qij (3,3)) of a density given at the quadrature points (T, 4)."""
        wr = self.wq * rho_q.ravel()
        y = self.yq
        Q = wr.sum()
        d = (wr[:, None] * y).sum(axis=0)
        r2 = (y * y).sum(axis=1)
        Qij = 3.0 * np.einsum("q,qi,qj->ij", wr, y, y) - np.eye(3) * (wr * r2).sum()
        return Q, d, Qij

    def boundary_values(self, rho_q):
        if self.lmax < 0:
            return np.zeros(len(self.Bd))
        Q, d, Qij = self.moments(rho_q)
        r = self.xyz[self.Bd] - self.center
        rn = np.sqrt((r * r).sum(axis=1))
        V = Q / rn
        if self.lmax >= 1:
            V = V + (r @ d) / rn ** 3
        if self.lmax >= 2:
            V = V + 0.5 * np.einsum("bi,ij,bj->b", r, Qij, r) / rn ** 5
        return V

    def _cg(self, b):
        x, info = spla.cg(self._L_II, b, x0=self._x, rtol=1e-13, atol=0.0, M=self._M, maxiter=100000)
        if info != 0:
            raise RuntimeError(f"Hartree CG did not converge (info={info})")
        self._x = x
        return x

    def solve(self, rho_q):
        """Nodal Hartree potential U (n_nodes,) for the density rho_q (T, 4)."""
        rhs = 4.0 * np.pi * fem.quad_to_nodes(rho_q, self.tet10, self.vol, self.n)
        U = np.zeros(self.n)
        U[self.Bd] = self.boundary_values(rho_q)
        U[self.I] = self.solve_II(rhs[self.I] - self.L_IB @ U[self.Bd])
        return U
