"""Learned preconditioner on the GPU against the oracle network (oracle/gcn.py).

Weights are drawn in Python and rounded to bfloat16-representable values, so the GPU's
bfloat16 use of them is exact and both sides evaluate the same network; float32 activations
on the GPU give relative agreement of ~1e-5 in the output and ~1e-3 in the gradients.
"""
import numpy as np
import pytest

from oracle import gcn, pcal
from paper_2007_14228_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ofks():
    from paper_2007_14228_gb300 import build
    build.build()
    from paper_2007_14228_gb300 import ofks as mod
    return mod


def bf16(x):
    """Round float32 values to the nearest bfloat16 (ties to even)."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def flat_to_params(w, width):
    dims = [gcn.N_FEAT, width, width, 1]
    out, o = [], 0
    for l in range(3):
        fi, fo = dims[l], dims[l + 1]
        W = w[o:o + fi * fo].reshape(fi, fo).astype(np.float64); o += fi * fo
        U = w[o:o + fi * fo].reshape(fi, fo).astype(np.float64); o += fi * fo
        b = w[o:o + fo].astype(np.float64); o += fo
        out.append({"W": W, "U": U, "b": b})
    return out


def setup(ofks, width, seed=0):
    s = I.lih().with_cells((8, 6, 6)).with_p(3, occ=1.0)
    m = I.make_mesh(s)
    ctx = ofks.context_for(s, m, beta=10.0, learned_tc=0)     # float32 activations for the oracle checks
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, s.Z, s.R, pcal.Params(p=3, occ=1.0, precond="exact",
                                                                          hartree=False, xc=False))
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((pr.n, 3))
    shifts = np.array([-0.9, -0.3, 0.2])
    ctx.precond_init(width, seed)
    w = ctx.precond_get_weights()
    w = bf16(0.3 * rng.standard_normal(w.size).astype(np.float32))
    ctx.precond_set_weights(w)
    A = gcn.mean_aggregator(gcn.dof_graph(m.tet10, m.dirichlet))
    return ctx, pr, G, shifts, w, A


@pytest.mark.parametrize("width", [8, 64])
def test_network_output_matches_oracle(ofks, width):
    ctx, pr, G, shifts, w, A = setup(ofks, width)
    D = ctx.precondition("learned", G, shifts)
    f, s, diag = gcn.features(G, pr.Lf.diagonal(), pr.Bf.diagonal(), shifts)
    Do, _, _ = gcn.predict(flat_to_params(w, width), f, s, A)
    Do[:, 2] = G[:, 2]                     # shift >= 0: T = I
    assert np.max(np.abs(D - Do)) < 2e-4 * np.max(np.abs(Do))
    ctx.close()


@pytest.mark.parametrize("width", [8, 64])
@pytest.mark.parametrize("kind", ["l2", "energy"])
def test_network_gradients_match_oracle(ofks, width, kind):
    ctx, pr, G, shifts, w, A = setup(ofks, width, seed=1)
    ctx.set_params(learned_loss=1 if kind == "energy" else 0)
    Dstar = pr.precondition(G, shifts)
    loss, g = ctx.precond_grads(G, shifts, Dstar)
    f, s, _ = gcn.features(G, pr.Lf.diagonal(), pr.Bf.diagonal(), shifts)
    params = flat_to_params(w, width)
    D, y, cache = gcn.predict(params, f, s, A)
    if kind == "energy":
        lo, dy = gcn.energy_loss_and_dy(D, Dstar, G, s, pr.Lf, pr.Bf, shifts)
    else:
        lo, dy = gcn.loss_and_dy(D, Dstar, s)
    grads = gcn.backward(params, cache, dy, A)
    go = np.concatenate([np.concatenate([gr["W"].ravel(), gr["U"].ravel(), gr["b"].ravel()]) for gr in grads])
    assert abs(loss - lo) < 1e-4 * lo
    assert np.max(np.abs(g - go)) < 1e-3 * np.max(np.abs(go)), np.max(np.abs(g - go)) / np.max(np.abs(go))
    ctx.close()


@pytest.mark.parametrize("kind,factor", [("l2", 0.75), ("energy", 0.92)])
def test_training_steps_reduce_the_loss(ofks, kind, factor):
    # 100 Adam steps on one pair from the Jacobi start (the energy-norm loss falls more slowly: it
    # weighs the smooth error the 3-hop network cannot reach; measured 0.549 -> 0.484)
    ctx, pr, G, shifts, w, A = setup(ofks, 16, seed=2)
    ctx.set_params(learned_loss=1 if kind == "energy" else 0)
    ctx.precond_init(16, 3)                 # last layer zero: starts as the Jacobi step
    Dstar = pr.precondition(G, shifts)
    losses = [ctx.train_precond_step(G, shifts, Dstar, lr=3e-3) for _ in range(100)]
    assert losses[-1] < factor * losses[0], (losses[0], losses[-1])
    ctx.close()


def test_learned_mode_keeps_the_fixed_point(ofks):
    # the judge and its PCG fallback make the learned mode change only the path
    s = I.lih().with_cells((6, 6, 6))
    m = I.make_mesh(s)
    V = I.initial_block(m.n_free, s.p, 0)
    E = {}
    for mode in ("pcg", "learned"):
        ctx = ofks.context_for(s, m, beta=10.0, tol=1e-10, max_iter=3000, precond=mode)
        if mode == "learned":
            ctx.precond_init(16, 5)
        ctx.init_orbitals(V)
        r = ctx.solve()
        E[mode] = r["e_total"]
        if mode == "learned":
            assert r["judge_total"] > 0
        ctx.close()
    assert abs(E["pcg"] - E["learned"]) < 1e-8


def test_tensor_core_layer_matches_cuda_cores(ofks):
    # the width-64 hidden layer on tcgen05 (bf16 operands, float32 accumulation in tensor memory)
    # against the float32 CUDA-core layer: agreement to bf16 rounding of the activations
    ctx, pr, G, shifts, w, A = setup(ofks, 64, seed=4)
    outs = {}
    for tc in (0, 1):
        ctx.set_params(p=3, occ=1.0, beta=10.0, learned_tc=tc)
        ctx.precond_set_weights(w)
        outs[tc] = ctx.precondition("learned", G, shifts)
    err = np.max(np.abs(outs[1] - outs[0])) / np.max(np.abs(outs[0]))
    assert err < 3e-2, err
    assert np.all(np.isfinite(outs[1]))
    ctx.close()


def test_trained_network_beats_the_jacobi_step_on_held_out_systems(ofks):
    # the committed weights (trained on seeds 1..150 by the library's own kernels) against the
    # untrained network, whose zero last layer makes it the Jacobi step, on pairs (G, T^-1 G)
    # from held-out random systems at iterations where multipliers are negative
    import os
    from paper_2007_14228_gb300 import train_precond as T
    w = np.load(os.path.join(os.path.dirname(ofks.__file__), "precond_weights.npy"))
    trained, jacobi = [], []
    for seed in (10005, 10006):
        for ctx, G, shifts, Dstar in T.pairs_from_system(seed, 14, (60, 120), None):
            ctx.precond_set_weights(w)
            trained.append(ctx.precond_grads(G, shifts, Dstar)[0])
            ctx.precond_init(64, seed)
            jacobi.append(ctx.precond_grads(G, shifts, Dstar)[0])
    assert trained and len(trained) == len(jacobi)
    # energy-norm errors (the default loss); on the training run's own held-out seeds 0.668 against 0.744
    assert np.mean(trained) < 0.95 * np.mean(jacobi), (np.mean(trained), np.mean(jacobi))


def read_pairs(path):
    """Parse a pairs file of ofks_record_pair: header (magic, n, p), then (shifts, G, D*) records."""
    raw = open(path, "rb").read()
    assert raw[:8] == b"OFKSPR1\x00"
    n = int(np.frombuffer(raw[8:16], np.int64)[0])
    p = int(np.frombuffer(raw[16:20], np.int32)[0])
    body = np.frombuffer(raw[24:], np.float64)
    rec = p + 2 * n * p
    assert body.size % rec == 0
    out = []
    for k in range(body.size // rec):
        r = body[k * rec:(k + 1) * rec]
        out.append((r[:p], r[p:p + n * p].reshape(n, p), r[p + n * p:].reshape(n, p)))
    return n, p, out


def test_pairs_recorded_and_trained_in_the_library(ofks, tmp_path):
    # ofks_record_pair appends (shifts, G, T^{-1} G) at the current iterate; the targets solve the
    # shifted systems of Eq. precondition-T with the oracle's own L and B; ofks_train_precond then
    # runs shuffled Adam epochs over the file and lowers the loss
    s = I.lih().with_cells((8, 8, 8))
    m = I.make_mesh(s)
    ctx = ofks.context_for(s, m, beta=10.0)
    ctx.precond_init(16, 3)
    ctx.init_orbitals(I.initial_block(m.n_free, s.p, 0))
    path = str(tmp_path / "pairs.bin")
    recorded = 0
    for _ in range(60):
        ctx.step(10)
        ctx.evaluate()
        if np.any(np.diag(ctx.get_field("Lambda")) < 0):
            assert ctx.record_pair(path) >= 1
            recorded += 1
            if recorded == 3:
                break
    assert recorded == 3
    n, p, pairs = read_pairs(path)
    assert (n, p) == (m.n_free, s.p) and len(pairs) == 3
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, s.Z, s.R, pcal.Params(p=s.p, occ=s.occ))
    for shifts, G, D in pairs:
        for c in range(p):
            if shifts[c] < 0:
                T = 0.5 * pr.Lf - shifts[c] * pr.Bf
                assert np.linalg.norm(T @ D[:, c] - G[:, c]) <= 1e-9 * np.linalg.norm(G[:, c])
            else:
                np.testing.assert_array_equal(D[:, c], G[:, c])
    loss1, st1 = ctx.train_precond(path, 1, 7)
    loss2, st2 = ctx.train_precond(path, 40, 7)
    assert st1 == 3 and st2 == 3 + 120
    assert loss2 < loss1
    # a pairs file belongs to one mesh and p: another shape is refused
    other = ofks.context_for(s.with_p(3, occ=1.0), m, beta=10.0)
    other.precond_init(16, 3)
    with pytest.raises(ofks.OfksError) as e:
        other.train_precond(path, 1, 0)
    assert e.value.code == ofks.EINVAL
    other.close()
    ctx.close()


def test_trained_network_keeps_the_fixed_point(ofks):
    # the learned form with the committed weights: the judge and the PCG fallback change the path
    # only; the converged energy and eigenvalues are those of the PCG form (LiH, 6^3 cells)
    s = I.lih().with_cells((6, 6, 6))
    m = I.make_mesh(s)
    V = I.initial_block(m.n_free, s.p, 0)
    out = {}
    for mode in ("pcg", "learned"):
        ctx = ofks.context_for(s, m, beta=10.0, tol=1e-11, max_iter=6000, precond=mode)
        if mode == "learned":
            ctx.precond_set_weights(ofks.trained_weights())
        ctx.init_orbitals(V)
        r = ctx.solve()
        assert r["converged"] == 1, mode
        out[mode] = (r["e_total"], ctx.rayleigh_ritz(), r["judge_total"])
        ctx.close()
    assert abs(out["pcg"][0] - out["learned"][0]) < 1e-8
    np.testing.assert_allclose(out["pcg"][1], out["learned"][1], atol=1e-7)
    assert out["learned"][2] > 0                  # the network was judged on every active column


def near_converged_lih(ofks):
    """LiH 6^3 solved to 1e-6 with the PCG: both multipliers are negative from here on, so every
    later direction preconditions two columns"""
    s = I.lih().with_cells((6, 6, 6))
    m = I.make_mesh(s)
    ctx = ofks.context_for(s, m, beta=10.0, tol=1e-6, max_iter=3000)
    ctx.init_orbitals(I.initial_block(m.n_free, s.p, 0))
    assert ctx.solve()["converged"] == 1
    assert np.all(np.diag(ctx.get_field("Lambda")) < 0)
    return ctx


def test_judge_accepts_takes_warm_starts_and_pauses_the_network(ofks):
    ctx = near_converged_lih(ofks)
    ctx.precond_init(16, 5)                  # zero last layer: the network is the Jacobi step M^-1 G
    w_jacobi = ctx.precond_get_weights()
    # (1) a judge that accepts every direction with G.D > 0 (M^-1 G always has it): the network runs
    # on every call and its directions are taken
    ctx.set_params(precond="learned", judge_tau=1e30, tol=1e-14)
    r = ctx.step(11)
    assert r["learned_calls"] == 11 and r["judge_total"] == 22 and r["judge_accept"] == 22
    # (2) a network far off (a large constant output): every column is rejected and, its residual
    # exceeding that of D = 0, started from zero; with no column taken the network pauses 1, 2, 4, ...
    # calls: it runs on calls 1, 3, 6 and 11 of the next 11
    w_bad = w_jacobi.copy()
    w_bad[-1] = 1e3                          # the output layer's bias
    ctx.precond_set_weights(w_bad)
    ctx.set_params(judge_tau=1e-30)
    r2 = ctx.step(11)
    assert r2["learned_calls"] - r["learned_calls"] == 4
    assert r2["judge_accept"] == r["judge_accept"] and r2["learned_warm"] == r["learned_warm"]
    # (3) learned_retry = 0: no pause
    ctx.set_params(learned_retry=0)
    r3 = ctx.step(5)
    assert r3["learned_calls"] - r2["learned_calls"] == 5
    assert np.isfinite(r3["e_total"])
    ctx.close()


def test_warm_started_pcg_matches_the_oracle_pcg_from_the_same_start(ofks):
    # a rejected column whose network residual is below that of zero runs the PCG from the network's
    # direction: D equals the oracle's Jacobi-PCG of Eq. precondition-T started from that direction
    ctx = near_converged_lih(ofks)
    ctx.precond_init(16, 5)                  # zero last layer: the network is the Jacobi step M^-1 G
    ctx.set_params(precond="learned", judge_tau=1e-30, tol=1e-14, pcg_iters=5)
    ctx.evaluate()
    G = ctx.get_field("G")
    lam = np.diag(ctx.get_field("Lambda")).copy()
    r0 = ctx.step(1)
    D = ctx.get_field("D")
    s = I.lih().with_cells((6, 6, 6))
    m = I.make_mesh(s)
    pr = pcal.Problem(m.xyz, m.tet10, m.dirichlet, s.Z, s.R, pcal.Params(p=s.p, occ=s.occ, pcg_iters=5))
    warm = 0
    for c in range(2):
        T = (0.5 * pr.Lf - lam[c] * pr.Bf).tocsr()
        Minv = 1.0 / T.diagonal()
        x = Minv * G[:, c]                   # the network's direction (the Jacobi step)
        r = G[:, c] - T @ x
        ratio = np.sqrt((r * Minv) @ r / ((G[:, c] * Minv) @ G[:, c]))
        if ratio >= 1.0:                     # not a better start than zero: the PCG starts from zero
            x = np.zeros_like(x)
            r = G[:, c].copy()
        else:
            warm += 1
        z = Minv * r
        pdir = z.copy()
        rz = r @ z
        for _ in range(5):
            q = T @ pdir
            a = rz / (pdir @ q)
            x += a * pdir
            r -= a * q
            z = Minv * r
            rzn = r @ z
            pdir = z + (rzn / rz) * pdir
            rz = rzn
        # the network's output is float32 (here M^-1 G rounded to float32), the PCG float64
        np.testing.assert_allclose(D[:, c], x, rtol=0, atol=1e-5 * np.max(np.abs(x)))
    assert r0["learned_warm"] == warm and warm >= 1, (r0, warm)
    ctx.close()


def test_trained_network_gains_over_the_method_without_it(ofks):
    # reduced chain (26 x 14 x 8 cells, n = 20,655, p = 41), float64, to (kkt + fea)/kkt0 < 1e-6 from
    # the same seeded start.  The committed network (i) alone, every direction taken, needs far fewer
    # iterations than no preconditioner (measured 731 against 3863: it is worth about two Jacobi-PCG
    # iterations), and (ii) as the start of the paper's PCG x8 for the columns the judge rejects, with
    # no pauses, keeps the PCG's iteration count (measured 221 and 234 with float32 and bf16 hidden
    # activations against 236: within the spread that rounding alone gives the BB path); every run
    # reaches the same energy
    s = I.chain(cells=(26, 14, 8))
    m = I.make_mesh(s)
    V = I.initial_block(m.n_free, s.p, 0)
    runs = {"none": dict(precond="none"), "alone": dict(precond="learned", judge_tau=1e30, learned_retry=0),
            "pcg": dict(precond="pcg"), "warm": dict(precond="learned", learned_retry=0)}
    out = {}
    for name, kw in runs.items():
        ctx = ofks.context_for(s, m, beta=10.0, tol=1e-6, max_iter=8000, **kw)
        if kw["precond"] == "learned":
            ctx.precond_set_weights(ofks.trained_weights())
        ctx.init_orbitals(V)
        r = ctx.solve()
        assert r["converged"] == 1, name
        out[name] = r
        ctx.close()
    assert out["alone"]["iters"] < 0.3 * out["none"]["iters"], (out["alone"]["iters"], out["none"]["iters"])
    assert out["warm"]["iters"] <= 1.05 * out["pcg"]["iters"], (out["warm"]["iters"], out["pcg"]["iters"])
    assert out["warm"]["learned_warm"] > 0
    for name in ("none", "alone", "warm"):      # the same fixed point, to this stopping tolerance
        assert abs(out[name]["e_total"] - out["pcg"]["e_total"]) < 1e-4, name
