"""PCAL for the FEM Kohn-Sham total-energy minimization (oracle, FP64).

Problem (Eq. prob:KS): minimize E_KS(X) subject to X^T B X = I_p, X in R^{n x p}, n the
free (interior) degrees of freedom of the P2 space with homogeneous Dirichlet data.

Pieces, in the paper's order and notation:
  density      rho = f tr(X^T calB X) evaluated at the quadrature points (Sec. 2.2);
               f is the occupation (electrons per orbital; the paper's Sec. 4.1 says two)
  potentials   V = V_ext (Eq. ext) + V_Har (FEM Poisson, Sec. 2.2) + V_xc (LDA)
  hamiltonian  H(X) = L/2 + M_ext + M_Har(X) + M_xc(X)  (Eq. hamiltonian)
  energy       E_KS = E_kin + E_ext + E_Har + E_xc + E_nuc  (Eq. totalEnergy and the
               discrete traces of Sec. 2.2), with occupation f on the density
  gradient     scaled to H(X) X (end of Sec. 2.2)
  iteration    Alg. 2 (PCAL, ``method='pcal'``):
                 Lambda0 = X^T H X                                    (Eq. multi)
                 Lambda  = Lambda0 + Theta(X^T grad L_beta(X, Lambda0)) (Eq. lambda2)
                 grad L_beta(X, Lambda) = H X - B X Lambda + beta B X (X^T B X - I)
                 D_i = T_i^{-1} grad_i L_beta with T_i = L/2 - Lambda_ii B if Lambda_ii < 0,
                       else I                                      (Eq. precondition-T)
                 X_i <- (X_i - D_i/eta) / ||X_i - D_i/eta||_B      (Eq. PCAL-main)
               Alg. 1 (PLAM, ``method='plam'``): Lambda = Lambda0 (Eq. multi), the shifts of
                 Eq. precondition-T from Lambda0, X <- X - D/eta without normalization
                 (Eq. PLAM-main)
               MOptQR (``method='moptqr'``, the manifold comparison method of Sec. 5): the
                 antigradient H X - B X Lambda0 on the B-Stiefel manifold, the same
                 preconditioner (shifts from Lambda0) and step size, then the step is put back on
                 the manifold by the Cholesky-based Gram-Schmidt of Sec. 4.2: Y^T B Y = R^T R,
                 X <- Y R^{-1}
  stopping     kkt = ||H X - B X Lambda0||_F, fea = ||X^T B X - I||_F,
               stop when (kkt + fea)/kkt_0 < tol (Sec. 4.1)
  step size    BB2 (Sec. 4.4) with S = X^k - X^{k-1}; Y is the difference of the directions
               actually applied (the preconditioned gradients), see ``Params.eta_rule``
  init         V = X0 R with R upper triangular (Cholesky-based Gram-Schmidt, Sec. 4.2)
  post         Rayleigh-Ritz on (X^T H X, X^T B X) and X <- X V (Sec. 4.3)

Readings where the paper is silent (shared with the CUDA path by specification only):
  * the preconditioned systems are solved by Jacobi-PCG from a zero guess with a fixed
    number of iterations (``pcg_iters``); an 'exact' mode iterates to 1e-12
  * eta_0 = ||D^0||_F / (1e-3 ||X^0||_F); eta is clamped to [eta_min, eta_max]; if
    <S, Y> = 0 the previous eta is kept
  * Lambda0 is symmetrized, sym(A) = (A + A^T)/2, to remove rounding asymmetry
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import dense, fem, xc
from .hartree import Hartree


@dataclass
class Params:
    p: int
    beta: float = 10.0
    occ: float = 2.0
    tol: float = 1e-8
    max_iter: int = 1000
    precond: str = "pcg"          # 'none' | 'pcg' | 'exact'
    pcg_iters: int = 8
    eta_rule: str = "bb2"         # 'bb2' | 'bb1' | 'abb1' | 'abb2' | 'bb2_raw' | 'fixed'
    method: str = "pcal"          # 'pcal' (Alg. 2) | 'plam' (Alg. 1) | 'moptqr' (Sec. 5)
    eta_fixed: float = 0.0        # used when eta_rule == 'fixed'
    eta_min: float = 1e-4
    eta_max: float = 1e8
    hartree: bool = True
    xc: bool = True
    multipole_lmax: int = 2


def nuclear_repulsion(Z, R) -> float:
    """E_nuc = sum_{j<k} Z_j Z_k / |R_j - R_k| (Sec. 2.1)."""
    e = 0.0
    for j in range(len(Z)):
        for k in range(j + 1, len(Z)):
            e += Z[j] * Z[k] / np.linalg.norm(R[j] - R[k])
    return float(e)


class Problem:
    """Discretized Kohn-Sham problem on one mesh (Sec. 2.2)."""

    def __init__(self, xyz, tet10, dirichlet, Z, R, params: Params):
        self.prm = params
        self.xyz, self.tet10 = np.asarray(xyz, np.float64), np.asarray(tet10, np.int64)
        self.dirichlet = np.asarray(dirichlet, np.uint8)
        self.Z, self.R = np.asarray(Z, np.float64), np.asarray(R, np.float64).reshape(-1, 3)
        self.n_nodes = self.xyz.shape[0]
        self.free = np.nonzero(self.dirichlet == 0)[0]
        self.n = len(self.free)
        L, B = fem.assemble_LB(self.xyz, self.tet10)
        self.L_full = L
        self.Lf = L[self.free][:, self.free].tocsr()
        self.Bf = B[self.free][:, self.free].tocsr()
        self.vol, _ = fem.tet_geometry(self.xyz, self.tet10)
        self.xq = fem.quad_points(self.xyz, self.tet10)   # (T, 4, 3)
        self.wq2 = np.repeat(self.vol[:, None] / 4.0, 4, axis=1)  # quadrature weights (T, 4)
        # V_ext at the quadrature points (Eq. ext); points are interior, never at a nucleus
        self.Vext_q = np.zeros(self.xq.shape[:2])
        for Zj, Rj in zip(self.Z, self.R):
            self.Vext_q -= Zj / np.sqrt(((self.xq - Rj) ** 2).sum(axis=2))
        self.E_nuc = nuclear_repulsion(self.Z, self.R)
        # potential matrices on the free DoFs: tet nodes mapped to free indices (-1 = Dirichlet)
        fidx = np.full(self.n_nodes, -1, dtype=np.int64)
        fidx[self.free] = np.arange(self.n)
        self._tetf = fidx[self.tet10]
        self._Nq = fem.basis_values(fem.quad_bary())       # (4, 10)
        rows = np.repeat(self._tetf, 10, axis=1).ravel()
        cols = np.tile(self._tetf, (1, 10)).ravel()
        keep = (rows >= 0) & (cols >= 0)
        self._keep = keep
        key = rows[keep] * self.n + cols[keep]
        uniq, self._pos = np.unique(key, return_inverse=True)
        self._indices = uniq % self.n
        self._indptr = np.searchsorted(uniq // self.n, np.arange(self.n + 1))
        self.hartree = (Hartree(self.xyz, self.tet10, self.dirichlet, self.L_full, self.vol, self.xq,
                                params.multipole_lmax) if params.hartree else None)

    # ------------------------------------------------------------------ fields

    def embed(self, X: np.ndarray) -> np.ndarray:
        """Free-DoF block (n, p) -> all nodes (n_nodes, p), zero on the Dirichlet boundary."""
        Xa = np.zeros((self.n_nodes,) + X.shape[1:])
        Xa[self.free] = X
        return Xa

    def density(self, X: np.ndarray) -> np.ndarray:
        """rho(x_q) = f sum_l psi_l(x_q)^2 with psi_l = X_l^T N (Sec. 2.2); shape (T, 4)."""
        psi = fem.values_at_quad(self.embed(X), self.tet10)   # (T, 4, p)
        return self.prm.occ * np.sum(psi * psi, axis=2)

    def potentials(self, rho_q: np.ndarray) -> dict:
        """V_ext + V_Har + V_xc at the quadrature points, with eps_xc and the Hartree field."""
        out = {"rho": rho_q, "Vext": self.Vext_q}
        if self.hartree is not None:
            U = self.hartree.solve(rho_q)
            out["U"] = U
            out["VH"] = fem.values_at_quad(U, self.tet10)
        else:
            out["U"] = np.zeros(self.n_nodes)
            out["VH"] = np.zeros_like(rho_q)
        if self.prm.xc:
            out["eps_xc"], out["Vxc"] = xc.lda(rho_q)
        else:
            out["eps_xc"], out["Vxc"] = np.zeros_like(rho_q), np.zeros_like(rho_q)
        out["V"] = out["Vext"] + out["VH"] + out["Vxc"]
        return out

    def potential_matrix(self, Vq: np.ndarray) -> sp.csr_matrix:
        """(M_V)_ij = sum_T sum_q (|T|/4) V(x_q) N_i(x_q) N_j(x_q) on the free DoFs."""
        w = self.wq2 * Vq
        local = np.einsum("tq,qa,qb->tab", w, self._Nq, self._Nq).ravel()[self._keep]
        data = np.bincount(self._pos, weights=local, minlength=len(self._indices))
        return sp.csr_matrix((data, self._indices, self._indptr), shape=(self.n, self.n))

    def hamiltonian(self, pot: dict) -> sp.csr_matrix:
        """H = L/2 + M_ext + M_Har + M_xc (Eq. hamiltonian)."""
        return (0.5 * self.Lf + self.potential_matrix(pot["V"])).tocsr()

    def energy(self, X: np.ndarray, pot: dict | None = None) -> dict:
        """E_KS components (Eq. totalEnergy) evaluated directly from their definitions."""
        if pot is None:
            pot = self.potentials(self.density(X))
        rho, w = pot["rho"], self.wq2
        e = {"kin": self.prm.occ * 0.5 * float(np.sum(X * (self.Lf @ X))),
             "ext": float(np.sum(w * pot["Vext"] * rho)),
             "har": 0.5 * float(np.sum(w * pot["VH"] * rho)),
             "xc": float(np.sum(w * pot["eps_xc"] * rho)),
             "nuc": self.E_nuc}
        e["total"] = e["kin"] + e["ext"] + e["har"] + e["xc"] + e["nuc"]
        return e

    # ------------------------------------------------------------------ init / post

    def initial_guess(self, V: np.ndarray) -> np.ndarray:
        """Cholesky-based Gram-Schmidt (Sec. 4.2): V^T B V = R^T R, X0 = V R^{-1}."""
        S = V.T @ (self.Bf @ V)
        Rt = np.linalg.cholesky(0.5 * (S + S.T))            # lower factor R^T
        return np.linalg.solve(Rt, V.T).T                   # V R^{-1} = (R^{-T} V^T)^T

    def rayleigh_ritz(self, X: np.ndarray):
        """Sec. 4.3: eigenpairs of (X^T H X) v = lam (X^T B X) v, then X <- X V."""
        pot = self.potentials(self.density(X))
        H = self.hamiltonian(pot)
        A = X.T @ (H @ X)
        S = X.T @ (self.Bf @ X)
        lam, V = dense.generalized_eigh(0.5 * (A + A.T), 0.5 * (S + S.T))
        return lam, X @ V

    # ------------------------------------------------------------------ preconditioner

    def precondition(self, G: np.ndarray, shifts: np.ndarray) -> np.ndarray:
        """D_i = T_i^{-1} G_i, T_i = L/2 - shift_i B for shift_i < 0, else D_i = G_i.

        Eq. (precondition-T).  Jacobi-preconditioned CG from a zero guess, every column an
        independent system; a fixed iteration count ('pcg') or to a 1e-12 relative residual
        ('exact').
        """
        D = G.copy()
        neg = np.nonzero(shifts < 0)[0]
        if self.prm.precond == "none" or len(neg) == 0:
            return D
        lam = shifts[neg]
        g = G[:, neg]
        dL, dB = self.Lf.diagonal(), self.Bf.diagonal()
        diag = 0.5 * dL[:, None] - lam[None, :] * dB[:, None]

        def T(P):
            return 0.5 * (self.Lf @ P) - (self.Bf @ P) * lam[None, :]

        x = np.zeros_like(g)
        r = g.copy()
        z = r / diag
        p = z.copy()
        rz = np.sum(r * z, axis=0)
        exact = self.prm.precond == "exact"
        r0 = np.linalg.norm(g, axis=0)
        iters = 10000 if exact else self.prm.pcg_iters
        for _ in range(iters):
            q = T(p)
            pq = np.sum(p * q, axis=0)
            alpha = np.where(pq > 0, rz / np.where(pq > 0, pq, 1.0), 0.0)
            x += alpha * p
            r -= alpha * q
            z = r / diag
            rz_new = np.sum(r * z, axis=0)
            beta = np.where(rz > 0, rz_new / np.where(rz > 0, rz, 1.0), 0.0)
            p = z + beta * p
            rz = rz_new
            if exact and np.all(np.linalg.norm(r, axis=0) <= 1e-12 * np.maximum(r0, 1e-300)):
                break
        D[:, neg] = x
        return D


@dataclass
class State:
    X: np.ndarray
    k: int = 0
    eta: float = 0.0
    kkt0: float = 0.0
    X_prev: np.ndarray | None = None
    D_prev: np.ndarray | None = None
    G_prev: np.ndarray | None = None
    history: list = field(default_factory=list)
    converged: bool = False


def sym(A):
    return 0.5 * (A + A.T)


def lagrangian_gradient(HX, BX, Lam, S, beta):
    """grad_X L_beta(X, Lambda) = H X - B X Lambda + beta B X (X^T B X - I).

    The gradient of the augmented Lagrangian of Eq. (ALM-sub) for symmetric Lambda, in the
    scaling of the end of Sec. 2.2 where the energy's gradient is H(X) X; S = X^T B X.
    """
    return HX - BX @ Lam + beta * BX @ (S - np.eye(S.shape[0]))


def theta(M):
    """Theta(M) = Diag(diag(M)) (notation of Sec. 1)."""
    return np.diag(np.diag(M))


def multipliers(X, HX, BX, Lam0, S, beta):
    """Eq. (lambda2): Lambda = Lambda0 + Theta(X^T grad_X L_beta(X, Lambda0)), Lambda0 = X^T H X."""
    return Lam0 + theta(X.T @ lagrangian_gradient(HX, BX, Lam0, S, beta))


def initial_eta(D0, X0):
    """eta_0 = ||D^0||_F / (1e-3 ||X^0||_F): the first step moves X by 1e-3 of its norm.

    The paper does not state eta_0; this is the reading taken.
    """
    return float(np.linalg.norm(D0) / (1e-3 * np.linalg.norm(X0)))


def step_size(rule, k, Sd, Yd, eta_prev):
    """eta_k of Sec. 4.4 from S = X^k - X^{k-1} and Y = the difference of the directions.

    BB1: |<S,Y>| / <S,S>;  BB2: <Y,Y> / |<S,Y>|;  ABB1: BB1 for odd k, BB2 for even k;
    ABB2: BB2 for odd k, BB1 for even k.  'bb2_raw' is BB2 (the caller passes raw-gradient
    differences).  When <S,Y> = 0 the previous eta is kept (a reading: the paper is silent).
    """
    sy, yy, ss = float(np.sum(Sd * Yd)), float(np.sum(Yd * Yd)), float(np.sum(Sd * Sd))
    if rule == "abb1":
        rule = "bb1" if k % 2 == 1 else "bb2"
    elif rule == "abb2":
        rule = "bb2" if k % 2 == 1 else "bb1"
    if sy == 0.0:
        return eta_prev
    if rule == "bb1":
        return abs(sy) / ss
    if rule in ("bb2", "bb2_raw"):
        return yy / abs(sy)
    raise ValueError(f"unknown eta rule {rule}")


def cholesky_qr(Y, BY):
    """Cholesky-based Gram-Schmidt (Sec. 4.2): Y^T B Y = R^T R, returns (Y R^{-1}, B Y R^{-1})."""
    S = Y.T @ BY
    Rt = np.linalg.cholesky(0.5 * (S + S.T))               # lower factor R^T
    return np.linalg.solve(Rt, Y.T).T, np.linalg.solve(Rt, BY.T).T


def iterate(prob: Problem, st: State) -> dict:
    """One pass of the loop body of Alg. 2 at X^k; updates st in place.

    Returns the record of iteration k: E, kkt, fea, eta and the p x p quantities.
    """
    prm = prob.prm
    X = st.X
    p = X.shape[1]
    I = np.eye(p)
    pot = prob.potentials(prob.density(X))
    H = prob.hamiltonian(pot)                              # H(X^k), Eq. hamiltonian
    HX = H @ X
    BX = prob.Bf @ X
    Lam0 = sym(X.T @ HX)                                   # Eq. multi
    S = X.T @ BX
    kkt = float(np.linalg.norm(HX - BX @ Lam0))            # ||(I - B X X^T) H X||_F
    fea = float(np.linalg.norm(S - I))
    E = prob.energy(X, pot)
    if st.k == 0:
        st.kkt0 = kkt
    rec = {"k": st.k, "E": E["total"], "kkt": kkt, "fea": fea, "Lambda0": Lam0, "S": S,
           "energy": E}
    if (kkt + fea) / st.kkt0 < prm.tol:
        st.converged = True
        rec["eta"] = st.eta
        st.history.append(rec)
        return rec
    method = prm.method
    if method == "pcal":
        # Eq. (lambda2) and the gradient of L_beta at Lambda
        Lam = multipliers(X, HX, BX, Lam0, S, prm.beta)
        G = lagrangian_gradient(HX, BX, Lam, S, prm.beta)
    elif method == "plam":
        # Alg. 1: the multipliers of Eq. (multi) in the gradient of Eq. (PLAM-main)
        Lam = Lam0
        G = lagrangian_gradient(HX, BX, Lam, S, prm.beta)
    elif method == "moptqr":
        # antigradient on the B-Stiefel manifold (no penalty: the iterates stay feasible)
        Lam = Lam0
        G = HX - BX @ Lam0
    else:
        raise ValueError(f"unknown method {method}")
    D = prob.precondition(G, np.diag(Lam))                 # Eq. (precondition-T)
    # step size (Sec. 4.4)
    if prm.eta_rule == "fixed":
        eta = prm.eta_fixed
    elif st.k == 0:
        eta = initial_eta(D, X)
    else:
        Yd = (G - st.G_prev) if prm.eta_rule == "bb2_raw" else (D - st.D_prev)
        eta = step_size(prm.eta_rule, st.k, X - st.X_prev, Yd, st.eta)
    eta = float(min(max(eta, prm.eta_min), prm.eta_max))
    Y = X - D / eta
    BY = prob.Bf @ Y
    if method == "pcal":
        # Eq. (PCAL-main): B-normalization of every column
        Xn = Y / np.sqrt(np.sum(Y * BY, axis=0))
    elif method == "plam":
        Xn = Y                                             # Eq. (PLAM-main)
    else:
        Xn, _ = cholesky_qr(Y, BY)
    st.X_prev, st.D_prev, st.G_prev = X, D, G
    st.X = Xn
    st.eta = eta
    st.k += 1
    rec.update({"eta": eta, "Lambda": Lam, "G": G, "D": D})
    st.history.append(rec)
    return rec


def solve(prob: Problem, X0: np.ndarray, max_iter: int | None = None, callback=None) -> State:
    """Alg. 2 from a feasible X0 until the stopping test holds or max_iter iterations."""
    st = State(X=X0.copy())
    limit = prob.prm.max_iter if max_iter is None else max_iter
    while True:
        rec = iterate(prob, st)
        if callback is not None:
            callback(rec)
        if st.converged or st.k >= limit:
            break
    return st
