"""Train the learned preconditioner on pairs the method itself generates.

For seeded random nuclei sets (4-12 nuclei, Z in {1, 6, 7, 8}, positions uniform in a 6 bohr
box, meshes of 16^3-24^3 cells) PCAL runs with the paper's PCG preconditioner; at sampled
iterations the library appends the pair (G, T^{-1} G) with the target solved to a tight residual
(ofks_record_pair) to a pairs file of that system, and then trains the network on the file
(ofks_train_precond: shuffled epochs of Adam steps of the library's own forward and backward
kernels).  This module only drives the systems and carries the weights from one system's
context to the next; the loop over pairs and steps runs in the library.

    python -m paper_2007_14228_gb300.train_precond --systems 100 --out weights.npy
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

from . import inputs as I
from . import ofks


def system_and_mesh(seed: int, cells: int):
    """A random nuclei set on the smallest grid of at least `cells` per axis that gives every
    segment between its anchors its two cells (many nuclei need more than the drawn size)."""
    for c in range(cells, cells + 40):
        s = I.random_nuclei(seed, cells=(c, c, c))
        try:
            return s, I.make_mesh(s)
        except ValueError:
            continue
    raise ValueError(f"no mesh for seed {seed}")


def pairs_from_system(seed: int, cells: int, samples, rng, device=0, width=64, weights=None):
    """Yield (ctx, G, shifts, Dstar) at the sampled iterations of one random system."""
    s, m = system_and_mesh(seed, cells)
    ctx = ofks.context_for(s, m, device=device, beta=10.0)
    if weights is not None:
        ctx.precond_set_weights(weights)
    else:
        ctx.precond_init(width, seed)
    ctx.init_orbitals(I.initial_block(m.n_free, s.p, seed))
    k = 0
    for target in samples:
        if target > k:
            ctx.step(target - k)
            k = target
        ctx.evaluate()
        G = ctx.get_field("G")
        shifts = np.diag(ctx.get_field("Lambda")).copy()
        if not np.any(shifts < 0):
            continue
        Dstar = ctx.precondition("exact", G, shifts)
        yield ctx, G, shifts, Dstar
    ctx.close()


def train(systems=100, first_seed=1, steps_per_pair=3, lr=1e-3, width=64,
          samples=(5, 10, 20, 30, 50, 80, 120, 160, 200, 250, 300),
          device=0, log=None, weights=None, workdir=None):
    """Pairs of each system go to a file of their own; the library trains on it for
    steps_per_pair epochs (one Adam step per pair and epoch, learning rate 1e-3)."""
    import tempfile
    if lr != 1e-3:
        raise ValueError("ofks_train_precond uses the learning rate 1e-3")
    rng = np.random.default_rng(first_seed)
    w = weights
    history = []
    n_pairs = 0
    t0 = time.time()
    tmp = workdir or tempfile.mkdtemp(prefix="ofks_pairs_")
    for seed in range(first_seed, first_seed + systems):
        cells = int(rng.integers(16, 25))
        s, m = system_and_mesh(seed, cells)
        ctx = ofks.context_for(s, m, device=device, beta=10.0)
        if w is not None:
            ctx.precond_set_weights(w)
        else:
            ctx.precond_init(width, seed)
        ctx.init_orbitals(I.initial_block(m.n_free, s.p, seed))
        path = os.path.join(tmp, f"pairs_{seed}.bin")
        k, recorded = 0, 0
        for target in samples:
            if target > k:
                ctx.step(target - k)
                k = target
            ctx.evaluate()
            if not np.any(np.diag(ctx.get_field("Lambda")) < 0):
                continue                       # every T = I: nothing to learn at this iterate
            n_pairs += ctx.record_pair(path)
            recorded += 1
        if recorded:
            loss, _ = ctx.train_precond(path, steps_per_pair, seed)
            history.append(loss)
            os.remove(path)
        w = ctx.precond_get_weights()
        ctx.close()
        if log:
            log({"system": seed, "cells": cells, "pairs": n_pairs, "loss": history[-1] if history else None,
                 "seconds": round(time.time() - t0, 1)})
    return w, history, n_pairs


def validate(weights, seeds, cells: int = 16, samples=(10, 30), device=0):
    """Mean loss of the network on pairs from held-out systems (no update)."""
    losses = []
    for seed in seeds:
        for ctx, G, shifts, Dstar in pairs_from_system(seed, cells, samples, None, device, weights=weights):
            loss, _ = ctx.precond_grads(G, shifts, Dstar)
            losses.append(loss)
    return float(np.mean(losses)) if losses else None


def evaluate(weights, seed: int, cells: int, device=0, tol=1e-6, max_iter=600):
    """Iterations to (kkt + fea)/kkt0 < tol with no preconditioner, the learned one and PCG."""
    s, m = system_and_mesh(seed, cells)
    V = I.initial_block(m.n_free, s.p, seed)
    out = {"seed": seed, "cells": cells, "p": s.p}
    for mode in ("none", "learned", "learned_unjudged", "pcg"):
        # learned_unjudged: every network direction with G.D > 0 is taken (the network alone)
        tau = 1e30 if mode == "learned_unjudged" else 0.5
        ctx = ofks.context_for(s, m, device=device, beta=10.0, tol=tol, max_iter=max_iter,
                               precond="learned" if mode.startswith("learned") else mode, judge_tau=tau)
        if mode.startswith("learned"):
            ctx.precond_set_weights(weights)
        ctx.init_orbitals(V)
        r = ctx.solve(allow_notconv=True)
        out[mode] = {"iters": r["iters"], "converged": r["converged"], "E": r["e_total"],
                     "accepted": r["judge_accept"], "judged": r["judge_total"]}
        ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--systems", type=int, default=100)
    ap.add_argument("--first-seed", type=int, default=1)
    ap.add_argument("--width", type=int, default=64)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--steps-per-pair", type=int, default=3)
    ap.add_argument("--out", default="precond_weights.npy")
    ap.add_argument("--eval-seed", type=int, default=10_000)
    ap.add_argument("--held-out", type=int, default=4, help="validation systems (seeds after the eval seed)")
    args = ap.parse_args()
    held = list(range(args.eval_seed + 1, args.eval_seed + 1 + args.held_out))
    w, hist, n = train(args.systems, args.first_seed, args.steps_per_pair, args.lr, args.width,
                       log=lambda d: print(json.dumps(d), flush=True))
    np.save(args.out, w)
    info = {"pairs": n, "systems": args.systems, "first_seed": args.first_seed, "width": args.width,
            "lr": args.lr, "steps_per_pair": args.steps_per_pair, "final_loss": hist[-1] if hist else None,
            "held_out_seeds": held, "held_out_loss": validate(w, held), "held_out_loss_jacobi": validate(None, held),
            "command": "python -m paper_2007_14228_gb300.train_precond " + " ".join(sys.argv[1:])}
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(info, f, indent=1)
    print(json.dumps(info), flush=True)
    print(json.dumps({"eval": evaluate(w, args.eval_seed, 16)}), flush=True)


if __name__ == "__main__":
    main()
