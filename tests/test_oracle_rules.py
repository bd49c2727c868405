"""Pins of the oracle's step-size rules, multipliers, Lagrangian gradient and comparison methods.

* BB rules (Sec. 4.4): with Y = A S for a symmetric positive definite A of known spectrum,
  eta^BB1 is the Rayleigh quotient of A at S and eta^BB2 the Rayleigh quotient of A at A^{1/2} S,
  so lambda_min <= BB1 <= BB2 <= lambda_max, both equal lambda at an eigenvector, and the
  alternating rules pick them by the parity of k.  The values are computed here from the
  eigen-decomposition of A, not from the dot products the oracle uses.
* Eq. (lambda2): at an iterate whose columns have unit B-norm but are not B-orthogonal, the
  multipliers make the column constraints stationary, diag(X^T grad L_beta(X, Lambda)) = 0
  (the diagonal multipliers D of Eq. kkt-PCAL vanish); Lambda0 alone does not.
* grad_X L_beta(X, Lambda) against central differences of L_beta(., Lambda) with Lambda held
  fixed (Eq. ALM-sub in the scaling where the energy's gradient is H X).
* PLAM (Alg. 1) and MOptQR (Sec. 5) reach the lowest eigenpairs of the dense pencil on a
  linear problem; MOptQR keeps every iterate feasible (X^T B X = I to rounding).

Each pin is a function that raises AssertionError; the tests below also plant plausible
mistakes in the oracle (swapped rules, a dropped or mis-signed Theta term, a wrong penalty
factor) and check that the pin catches each of them.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import pcal
from paper_2007_14228_gb300 import inputs as I


# ------------------------------------------------------------------------------ step sizes

def _spd(n, lo, hi, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.sort(rng.uniform(lo, hi, n))
    lam[0], lam[-1] = lo, hi
    return Q, lam


def check_bb_rules():
    n, p = 24, 3
    Q, lam = _spd(n * p, 0.5, 40.0, 3)
    A = (Q * lam) @ Q.T
    rng = np.random.default_rng(8)
    Sd = rng.standard_normal((n, p))
    Yd = (A @ Sd.ravel()).reshape(n, p)
    c2 = (Q.T @ Sd.ravel()) ** 2                     # squared coordinates in the eigenbasis
    bb1 = np.sum(c2 * lam) / np.sum(c2)
    bb2 = np.sum(c2 * lam ** 2) / np.sum(c2 * lam)
    got1 = pcal.step_size("bb1", 5, Sd, Yd, -1.0)
    got2 = pcal.step_size("bb2", 5, Sd, Yd, -1.0)
    assert abs(got1 - bb1) <= 1e-12 * bb1, (got1, bb1)
    assert abs(got2 - bb2) <= 1e-12 * bb2, (got2, bb2)
    assert lam[0] <= got1 <= got2 <= lam[-1]
    # the paper takes |<S, Y>|: negative curvature gives the same eta
    assert pcal.step_size("bb1", 5, Sd, -Yd, -1.0) == pytest.approx(bb1, rel=1e-12)
    assert pcal.step_size("bb2", 5, Sd, -Yd, -1.0) == pytest.approx(bb2, rel=1e-12)
    # at an eigenvector both rules return its eigenvalue
    v = Q[:, 7].reshape(n, p)
    Av = (A @ v.ravel()).reshape(n, p)
    assert pcal.step_size("bb1", 2, v, Av, -1.0) == pytest.approx(lam[7], rel=1e-10)
    assert pcal.step_size("bb2", 2, v, Av, -1.0) == pytest.approx(lam[7], rel=1e-10)
    # alternating rules: ABB1 = BB1 on odd k, BB2 on even k; ABB2 the other way round
    for k in (1, 2, 3, 4):
        odd = k % 2 == 1
        assert pcal.step_size("abb1", k, Sd, Yd, -1.0) == pytest.approx(bb1 if odd else bb2, rel=1e-12)
        assert pcal.step_size("abb2", k, Sd, Yd, -1.0) == pytest.approx(bb2 if odd else bb1, rel=1e-12)
    # <S, Y> = 0: the previous eta is kept
    Y0 = np.zeros_like(Sd)
    Y0[0, 0], Y0[1, 0] = Sd[1, 0], -Sd[0, 0]
    Sz = np.zeros_like(Sd)
    Sz[:2, 0] = Sd[:2, 0]
    assert pcal.step_size("bb2", 3, Sz, Y0, 7.25) == 7.25


def test_bb_rules_are_rayleigh_quotients_of_the_curvature():
    check_bb_rules()


@pytest.mark.parametrize("mistake", ["swap_bb", "swap_parity", "no_abs"])
def test_bb_pin_catches_planted_mistakes(monkeypatch, mistake):
    true = pcal.step_size

    def planted(rule, k, Sd, Yd, eta_prev):
        if mistake == "swap_bb" and rule in ("bb1", "bb2"):
            rule = {"bb1": "bb2", "bb2": "bb1"}[rule]
        if mistake == "swap_parity" and rule in ("abb1", "abb2"):
            k += 1
        if mistake == "no_abs":
            sy = float(np.sum(Sd * Yd))
            if rule == "bb1":
                return sy / float(np.sum(Sd * Sd))
            if rule == "bb2":
                return float(np.sum(Yd * Yd)) / sy
        return true(rule, k, Sd, Yd, eta_prev)

    monkeypatch.setattr(pcal, "step_size", planted)
    with pytest.raises(AssertionError):
        check_bb_rules()


def test_initial_step_moves_x_by_one_thousandth():
    # the reading of eta_0: the first (unnormalized) step X0 - D/eta0 has length 1e-3 ||X0||
    s = I.lih().with_cells((6, 4, 4))
    m = I.make_mesh(s)
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, s.Z, s.R, pcal.Params(p=s.p, occ=s.occ))
    st = pcal.State(X=pr.initial_guess(I.initial_block(pr.n, s.p, 0)))
    X0 = st.X.copy()
    rec = pcal.iterate(pr, st)
    assert np.linalg.norm(rec["D"] / rec["eta"]) == pytest.approx(1e-3 * np.linalg.norm(X0), rel=1e-12)


# ------------------------------------------------------------------------------ multipliers

@pytest.fixture(scope="module")
def lih_unit_columns():
    """An iterate of LiH (6x4x4 cells, p = 3) with unit B-norm columns that are not B-orthogonal."""
    s = I.lih().with_cells((6, 4, 4)).with_p(3)
    m = I.make_mesh(s)
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, s.Z, s.R, pcal.Params(p=3, occ=s.occ, beta=10.0))
    rng = np.random.default_rng(21)
    X = pr.initial_guess(I.initial_block(pr.n, 3, 0)) + 0.3 * rng.standard_normal((pr.n, 3)) / np.sqrt(pr.n)
    X = X / np.sqrt(np.sum(X * (pr.Bf @ X), axis=0))
    return pr, X


def check_multipliers(pr, X):
    H = pr.hamiltonian(pr.potentials(pr.density(X)))
    HX, BX = H @ X, pr.Bf @ X
    S = X.T @ BX
    assert np.max(np.abs(np.diag(S) - 1.0)) < 1e-13 and np.linalg.norm(S - np.eye(3)) > 1e-2
    Lam0 = pcal.sym(X.T @ HX)
    beta = pr.prm.beta
    Lam = pcal.multipliers(X, HX, BX, Lam0, S, beta)
    # only the diagonal changes (Theta), and the column constraints become stationary
    off = ~np.eye(3, dtype=bool)
    assert np.array_equal(Lam[off], Lam0[off])
    scale = np.max(np.abs(Lam0))
    d = np.diag(X.T @ pcal.lagrangian_gradient(HX, BX, Lam, S, beta))
    assert np.max(np.abs(d)) < 1e-11 * scale, d
    d0 = np.diag(X.T @ pcal.lagrangian_gradient(HX, BX, Lam0, S, beta))
    assert np.max(np.abs(d0)) > 1e-4 * scale            # Lambda0 alone leaves them non-stationary


def test_multipliers_make_the_column_constraints_stationary(lih_unit_columns):
    check_multipliers(*lih_unit_columns)


@pytest.mark.parametrize("mistake", ["full_matrix", "wrong_sign", "dropped"])
def test_multiplier_pin_catches_planted_mistakes(monkeypatch, lih_unit_columns, mistake):
    def planted(X, HX, BX, Lam0, S, beta):
        M = X.T @ pcal.lagrangian_gradient(HX, BX, Lam0, S, beta)
        if mistake == "full_matrix":
            return Lam0 + M
        if mistake == "wrong_sign":
            return Lam0 - pcal.theta(M)
        return Lam0

    monkeypatch.setattr(pcal, "multipliers", planted)
    with pytest.raises(AssertionError):
        check_multipliers(*lih_unit_columns)


def check_lagrangian_gradient(pr, X):
    # L_beta(X, Lambda) = E(X)/(2f) - <Lambda, X^T B X - I>/2 + beta/4 ||X^T B X - I||^2, Lambda fixed
    rng = np.random.default_rng(5)
    p = X.shape[1]
    A = rng.standard_normal((p, p))
    Lam = 0.5 * (A + A.T)
    beta, f, Ip = pr.prm.beta, pr.prm.occ, np.eye(p)

    def merit(Y):
        S = Y.T @ (pr.Bf @ Y)
        return pr.energy(Y)["total"] / (2 * f) - 0.5 * np.sum(Lam * (S - Ip)) + beta / 4 * np.sum((S - Ip) ** 2)

    Zd = rng.standard_normal(X.shape)
    h = 1e-5
    fd = (merit(X + h * Zd) - merit(X - h * Zd)) / (2 * h)
    H = pr.hamiltonian(pr.potentials(pr.density(X)))
    G = pcal.lagrangian_gradient(H @ X, pr.Bf @ X, Lam, X.T @ (pr.Bf @ X), beta)
    an = float(np.sum(Zd * G))
    assert abs(fd - an) < 1e-6 * abs(an), (fd, an)


@pytest.fixture(scope="module")
def lih_zero_boundary():
    # homogeneous Hartree boundary data: the Hartree term's gradient is then exactly M_H X (Sec. 2.2)
    s = I.lih().with_cells((6, 4, 4))
    m = I.make_mesh(s)
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, s.Z, s.R,
                      pcal.Params(p=s.p, occ=s.occ, beta=10.0, multipole_lmax=-1))
    rng = np.random.default_rng(13)
    X = pr.initial_guess(I.initial_block(pr.n, s.p, 1)) * 1.1 + 0.05 * rng.standard_normal((pr.n, s.p))
    return pr, X


def test_lagrangian_gradient_by_central_differences(lih_zero_boundary):
    check_lagrangian_gradient(*lih_zero_boundary)


@pytest.mark.parametrize("mistake", ["penalty_sign", "penalty_factor", "multiplier_side"])
def test_lagrangian_gradient_pin_catches_planted_mistakes(monkeypatch, lih_zero_boundary, mistake):
    def planted(HX, BX, Lam, S, beta):
        Ip = np.eye(S.shape[0])
        if mistake == "penalty_sign":
            return HX - BX @ Lam - beta * BX @ (S - Ip)
        if mistake == "penalty_factor":
            return HX - BX @ Lam + 0.5 * beta * BX @ (S - Ip)
        # the multiplier term without the 1/2 of <Lambda, X^T B X - I>/2
        return HX - 2.0 * BX @ Lam + beta * BX @ (S - Ip)

    monkeypatch.setattr(pcal, "lagrangian_gradient", planted)
    with pytest.raises(AssertionError):
        check_lagrangian_gradient(*lih_zero_boundary)


# ------------------------------------------------------------------------------ PLAM, MOptQR

@pytest.mark.parametrize("method", ["plam", "moptqr"])
def test_comparison_methods_reach_the_dense_eigenpairs(method):
    s = I.lih().with_cells((6, 6, 6)).with_p(3)
    m = I.make_mesh(s)
    prm = pcal.Params(p=3, occ=s.occ, hartree=False, xc=False, beta=10.0, tol=1e-11, max_iter=3000,
                      method=method)
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, s.Z, s.R, prm)
    st = pcal.solve(pr, pr.initial_guess(I.initial_block(pr.n, 3, 0)))
    assert st.converged
    lam, _ = pr.rayleigh_ritz(st.X)
    H = pr.hamiltonian(pr.potentials(np.zeros_like(pr.Vext_q))).toarray()
    ref = sla.eigh(H, pr.Bf.toarray(), eigvals_only=True, subset_by_index=[0, 2])
    np.testing.assert_allclose(lam, ref, atol=1e-9)
    if method == "moptqr":
        # the Cholesky-based Gram-Schmidt puts every iterate back on the manifold
        assert max(r["fea"] for r in st.history) < 1e-13
    else:
        # PLAM's iterates are infeasible on the way and feasible at the end
        assert max(r["fea"] for r in st.history) > 1e-3 and st.history[-1]["fea"] < 1e-9
