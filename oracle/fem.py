"""P2 finite elements on tetrahedra: basis, quadrature and assembly (oracle).

Follows Sec. 2.2 of the paper: the space V_h with basis phi_i, the mass matrix
B_ij = int phi_i phi_j, the stiffness L_ij = int grad phi_i . grad phi_j and the
potential matrices (M_V)_ij = int V phi_i phi_j (Eq. hamiltonian).  The paper uses
linear elements; the formulas are independent of the element order and are applied
here to quadratic (P2) elements.

Local numbering: vertices 0..3, then midpoints of edges 01, 02, 03, 12, 13, 23.
With barycentric coordinates lam_k:
    N_a  = lam_a (2 lam_a - 1)            (vertex a)
    N_ab = 4 lam_a lam_b                  (edge ab)
Quadrature for potential and density terms: the symmetric 4-point rule (degree 2),
points with barycentric (qa, qb, qb, qb) and permutations, weights |T|/4.
L is integrated with the same rule (its integrand has degree 2, so this is exact);
B is integrated exactly with int lam^alpha = 6|T| alpha! / (|alpha| + 3)!.
"""
from __future__ import annotations

from math import factorial

import numpy as np
import scipy.sparse as sp

EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
QA = (5.0 + 3.0 * np.sqrt(5.0)) / 20.0
QB = (5.0 - np.sqrt(5.0)) / 20.0


def quad_bary() -> np.ndarray:
    """(4, 4) barycentric coordinates of the 4 quadrature points (row q: point q)."""
    lam = np.full((4, 4), QB)
    np.fill_diagonal(lam, QA)
    return lam


def basis_values(lam: np.ndarray) -> np.ndarray:
    """P2 basis values at barycentric points lam (..., 4) -> (..., 10)."""
    out = np.empty(lam.shape[:-1] + (10,))
    for a in range(4):
        out[..., a] = lam[..., a] * (2.0 * lam[..., a] - 1.0)
    for e, (a, b) in enumerate(EDGES):
        out[..., 4 + e] = 4.0 * lam[..., a] * lam[..., b]
    return out


def basis_gradients(lam: np.ndarray, glam: np.ndarray) -> np.ndarray:
    """Gradients of the P2 basis.

    lam  (Q, 4) barycentric coordinates of Q points (same for every tet)
    glam (T, 4, 3) gradients of the barycentric coordinates of T tets
    returns (T, Q, 10, 3)
    """
    T, Q = glam.shape[0], lam.shape[0]
    g = np.empty((T, Q, 10, 3))
    for a in range(4):
        g[:, :, a, :] = (4.0 * lam[None, :, a, None] - 1.0) * glam[:, None, a, :]
    for e, (a, b) in enumerate(EDGES):
        g[:, :, 4 + e, :] = 4.0 * (lam[None, :, a, None] * glam[:, None, b, :]
                                   + lam[None, :, b, None] * glam[:, None, a, :])
    return g


def tet_geometry(xyz: np.ndarray, tet10: np.ndarray):
    """Volumes |T| (T,) and barycentric gradients (T, 4, 3) of straight-sided tets."""
    P = xyz[tet10[:, :4]]                                  # (T, 4, 3)
    J = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2)  # columns
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)                                # rows = grad lam_1..3
    glam = np.empty((len(tet10), 4, 3))
    glam[:, 1:, :] = Jinv
    glam[:, 0, :] = -Jinv.sum(axis=1)
    return np.abs(det) / 6.0, glam


def quad_points(xyz: np.ndarray, tet10: np.ndarray) -> np.ndarray:
    """Physical quadrature points (T, 4, 3): x_q = sum_k lam_k(q) P_k."""
    P = xyz[tet10[:, :4]]
    return np.einsum("qk,tkd->tqd", quad_bary(), P)


def _monomials_p2():
    """Each P2 basis function as {exponent tuple (4,): coefficient} in barycentric monomials."""
    polys = []
    for a in range(4):
        e2 = [0, 0, 0, 0]; e2[a] = 2
        e1 = [0, 0, 0, 0]; e1[a] = 1
        polys.append({tuple(e2): 2.0, tuple(e1): -1.0})
    for a, b in EDGES:
        e = [0, 0, 0, 0]; e[a] = 1; e[b] = 1
        polys.append({tuple(e): 4.0})
    return polys


def reference_mass() -> np.ndarray:
    """(10, 10) matrix with B_local = |T| * reference_mass(), integrated exactly.

    int_T lam^alpha dx = 6 |T| alpha_0! alpha_1! alpha_2! alpha_3! / (|alpha| + 3)!
    """
    polys = _monomials_p2()
    M = np.zeros((10, 10))
    for i in range(10):
        for j in range(10):
            s = 0.0
            for ei, ci in polys[i].items():
                for ej, cj in polys[j].items():
                    al = [x + y for x, y in zip(ei, ej)]
                    num = 6.0 * np.prod([factorial(x) for x in al])
                    s += ci * cj * num / factorial(sum(al) + 3)
            M[i, j] = s
    return M


def _scatter(n, tet10, local):
    """Sum local (T, 10, 10) matrices into an n x n CSR matrix."""
    rows = np.repeat(tet10, 10, axis=1).ravel()
    cols = np.tile(tet10, (1, 10)).ravel()
    A = sp.coo_matrix((local.ravel(), (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


def assemble_LB(xyz: np.ndarray, tet10: np.ndarray, chunk: int = 200_000):
    """Stiffness L and mass B over all nodes (Sec. 2.2), as CSR."""
    n = xyz.shape[0]
    lam = quad_bary()
    Bref = reference_mass()
    L = sp.csr_matrix((n, n))
    B = sp.csr_matrix((n, n))
    for s in range(0, len(tet10), chunk):
        t = tet10[s:s + chunk]
        vol, glam = tet_geometry(xyz, t)
        g = basis_gradients(lam, glam)                     # (T, 4, 10, 3)
        Lloc = np.einsum("t,tqad,tqbd->tab", vol / 4.0, g, g)
        Bloc = vol[:, None, None] * Bref[None]
        L = L + _scatter(n, t, Lloc)
        B = B + _scatter(n, t, Bloc)
    return L.tocsr(), B.tocsr()


class PotentialAssembler:
    """Assembly of (M_V)_ij = sum_T sum_q (|T|/4) V(x_q) N_i(x_q) N_j(x_q) (Eq. hamiltonian).

    The sparsity pattern of the full-node matrix is fixed by the mesh, so the CSR
    structure is built once and each assembly sums the local entries into it.
    """

    def __init__(self, n: int, tet10: np.ndarray, vol: np.ndarray):
        self.n = n
        self.vol = vol
        self.Nq = basis_values(quad_bary())                # (4, 10)
        rows = np.repeat(tet10, 10, axis=1).ravel()
        cols = np.tile(tet10, (1, 10)).ravel()
        key = rows.astype(np.int64) * n + cols
        uniq, self.pos = np.unique(key, return_inverse=True)
        self.indices = (uniq % n).astype(np.int64)
        r = uniq // n
        self.indptr = np.searchsorted(r, np.arange(n + 1)).astype(np.int64)

    def assemble(self, Vq: np.ndarray) -> sp.csr_matrix:
        """Vq (T, 4) potential at the quadrature points of every tet."""
        w = (self.vol[:, None] / 4.0) * Vq                 # (T, 4)
        local = np.einsum("tq,qa,qb->tab", w, self.Nq, self.Nq)
        data = np.bincount(self.pos, weights=local.ravel(), minlength=len(self.indices))
        return sp.csr_matrix((data, self.indices, self.indptr), shape=(self.n, self.n))


def values_at_quad(U_nodes: np.ndarray, tet10: np.ndarray) -> np.ndarray:
    """Evaluate a nodal field (n_nodes,) or block (n_nodes, p) at the quadrature points.

    psi(x_q) = sum_i U_i N_i(x_q) -> (T, 4) or (T, 4, p)
    """
    Nq = basis_values(quad_bary())                         # (4, 10)
    if U_nodes.ndim == 1:
        return np.einsum("qa,ta->tq", Nq, U_nodes[tet10])
    return np.einsum("qa,tal->tql", Nq, U_nodes[tet10])


def quad_to_nodes(fq: np.ndarray, tet10: np.ndarray, vol: np.ndarray, n: int) -> np.ndarray:
    """Load vector b_i = sum_T sum_q (|T|/4) f(x_q) N_i(x_q)."""
    Nq = basis_values(quad_bary())
    local = np.einsum("tq,qa->ta", (vol[:, None] / 4.0) * fq, Nq)
    return np.bincount(tet10.ravel(), weights=local.ravel(), minlength=n)
