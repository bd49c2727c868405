"""Learned preconditioner network (oracle, float64): features, forward, loss and backward.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper's preconditioner is D_i = T_i^{-1} G_i with T_i = L/2 - Lambda_ii B (Eq. precondition-T).
The learned stand-in maps a gradient column to an approximate T_i^{-1} G_i with a small graph
network on the free-DoF graph of the P2 mesh (one node per free degree of freedom, an edge
between two DoFs that share a tetrahedron: the structural pattern of L, which keeps the entries
of the stiffness that happen to vanish for right-angled elements).  Everything here is written out plainly so that the GPU kernels'
values and gradients can be checked against it.

Per column c with shift lam_c (lam_c = Lambda_cc if negative, else 0):
    diag_i  = dL_i / 2 - lam_c dB_i                      (Jacobi diagonal of T_c)
    z_i     = g_i / diag_i                                (one Jacobi step)
    s_c     = sqrt(mean_i z_i^2)                          (column scale)
    features f = [z_i / s_c,  log diag_i - mean_i log diag_i,  -lam_c dB_i / diag_i,  1]
Aggregation A: mean over the closed neighbourhood, (A h)_i = sum_{j in N(i)} h_j / |N(i)|.
Layers (widths 4 -> H -> H -> 1):  Z_l = H_l W_l + (A H_l) U_l + b_l,  H_{l+1} = relu(Z_l) for the
two hidden layers, identity for the last.
Output: D_i = s_c (f0_i + H_3,i)   (the network corrects the scaled Jacobi step).
Loss over a batch of columns, one of two:
    "l2":     mean over all columns of ||D_c - D*_c||^2 / ||D*_c||^2
    "energy": mean over the columns with a negative shift of
              (D_c - D*_c)^T T_c (D_c - D*_c) / (G_c^T D*_c)
the error in the energy norm of T_c (the norm the conjugate-gradient method of Eq. precondition-T
reduces, so a network direction is worth as much as a PCG iterate of the same energy error; the
plain l2 error leaves high-frequency errors almost free, which the residual T D - G amplifies),
relative to the energy norm of the exact solution, ||D*_c||_T^2 = G_c^T T_c^{-1} G_c = G_c^T D*_c.
Columns with a non-negative shift have T = I in Eq. precondition-T and are not preconditioned by
the network in the solver, so the energy loss leaves them out.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

N_FEAT = 4


def dof_graph(tet10: np.ndarray, dirichlet: np.ndarray) -> sp.csr_matrix:
    """Free-DoF adjacency of the mesh: ones where two free DoFs share a tetrahedron (and on the
    diagonal), whatever the values of L there."""
    free = np.cumsum(dirichlet == 0) - 1
    free[dirichlet != 0] = -1
    T = free[tet10]
    r = np.repeat(T, T.shape[1], axis=1).ravel()
    c = np.tile(T, (1, T.shape[1])).ravel()
    keep = (r >= 0) & (c >= 0)
    n = int(np.sum(dirichlet == 0))
    G = sp.csr_matrix((np.ones(int(keep.sum())), (r[keep], c[keep])), shape=(n, n))
    G.data[:] = 1.0
    return G


def mean_aggregator(pattern: sp.csr_matrix) -> sp.csr_matrix:
    """A with A_ij = 1/|N(i)| on the sparsity pattern (closed neighbourhoods)."""
    P = pattern.tocsr(copy=True)
    P.data = np.ones_like(P.data)
    deg = np.diff(P.indptr)
    return sp.diags(1.0 / deg) @ P


def features(G: np.ndarray, dL: np.ndarray, dB: np.ndarray, shifts: np.ndarray):
    """Input features (n, p, 4), the column scales s (p,) and the Jacobi diagonals (n, p)."""
    lam = np.where(shifts < 0, shifts, 0.0)
    diag = 0.5 * dL[:, None] - lam[None, :] * dB[:, None]
    z = G / diag
    s = np.sqrt(np.mean(z * z, axis=0))
    logd = np.log(diag)
    f = np.empty(G.shape + (N_FEAT,))
    f[..., 0] = z / s
    f[..., 1] = logd - logd.mean(axis=0)
    f[..., 2] = -lam[None, :] * dB[:, None] / diag
    f[..., 3] = 1.0
    return f, s, diag


def init_params(width: int = 64, seed: int = 0):
    """He-initialized weights; the last layer starts at zero (the network starts as Jacobi)."""
    rng = np.random.default_rng(seed)
    dims = [N_FEAT, width, width, 1]
    params = []
    for l in range(3):
        fi, fo = dims[l], dims[l + 1]
        sc = 0.0 if l == 2 else np.sqrt(2.0 / (2 * fi))
        params.append({"W": rng.standard_normal((fi, fo)) * sc, "U": rng.standard_normal((fi, fo)) * sc,
                       "b": np.zeros(fo)})
    return params


def forward(params, f: np.ndarray, A: sp.csr_matrix):
    """f (n, p, F0) -> y (n, p) network output, with the cache for backward."""
    n, p, _ = f.shape
    H = f
    cache = []
    for l, P in enumerate(params):
        AH = np.stack([A @ H[:, c, :] for c in range(p)], axis=1)     # per column, over nodes
        Z = H @ P["W"] + AH @ P["U"] + P["b"]
        cache.append((H, AH, Z))
        H = np.maximum(Z, 0.0) if l < 2 else Z
    return H[..., 0], cache


def predict(params, f, s, A):
    y, cache = forward(params, f, A)
    return s[None, :] * (f[..., 0] + y), y, cache


def loss_and_dy(D: np.ndarray, Dstar: np.ndarray, s: np.ndarray):
    """Relative squared error averaged over columns and its gradient with respect to y."""
    den = np.sum(Dstar * Dstar, axis=0)
    r = D - Dstar
    p = D.shape[1]
    loss = float(np.mean(np.sum(r * r, axis=0) / den))
    dD = 2.0 * r / den[None, :] / p
    return loss, dD * s[None, :]


def energy_loss_and_dy(D: np.ndarray, Dstar: np.ndarray, G: np.ndarray, s: np.ndarray, L: sp.spmatrix,
                       B: sp.spmatrix, shifts: np.ndarray):
    """Energy-norm error averaged over the columns with a negative shift, and its gradient with
    respect to y: with E_c = D_c - D*_c and T_c = L/2 - shift_c B,
    loss = mean_c E_c^T T_c E_c / (G_c^T D*_c),  dloss/dD_c = 2 T_c E_c / (G_c^T D*_c) / n_active."""
    act = shifts < 0
    na = int(act.sum())
    dD = np.zeros_like(D)
    if na == 0:
        return 0.0, dD
    loss = 0.0
    for c in np.nonzero(act)[0]:
        E = D[:, c] - Dstar[:, c]
        TE = 0.5 * (L @ E) - shifts[c] * (B @ E)
        den = float(G[:, c] @ Dstar[:, c])
        loss += float(E @ TE) / den
        dD[:, c] = 2.0 * TE / den / na
    return loss / na, dD * s[None, :]


def backward(params, cache, dy: np.ndarray, A: sp.csr_matrix):
    """Gradients of the loss for every W, U, b given dL/dy (n, p)."""
    n, p = dy.shape
    AT = A.T.tocsr()
    grads = [None] * 3
    dH = dy[..., None]
    for l in range(2, -1, -1):
        H, AH, Z = cache[l]
        dZ = dH if l == 2 else dH * (Z > 0)
        P = params[l]
        gW = np.einsum("ncf,nco->fo", H, dZ)
        gU = np.einsum("ncf,nco->fo", AH, dZ)
        gb = dZ.sum(axis=(0, 1))
        grads[l] = {"W": gW, "U": gU, "b": gb}
        dAH = dZ @ P["U"].T
        dH = dZ @ P["W"].T + np.stack([AT @ dAH[:, c, :] for c in range(p)], axis=1)
    return grads


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update in place; state holds the moments and the step count."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for l in range(3):
        for k in ("W", "U", "b"):
            key = (l, k)
            m = state.setdefault(("m",) + key, np.zeros_like(params[l][k]))
            v = state.setdefault(("v",) + key, np.zeros_like(params[l][k]))
            g = grads[l][k]
            m[:] = b1 * m + (1 - b1) * g
            v[:] = b2 * v + (1 - b2) * g * g
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            params[l][k] = params[l][k] - lr * mh / (np.sqrt(vh) + eps)
    return params
