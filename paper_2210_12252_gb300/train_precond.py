"""Train the learned per-mode preconditioner on the GPU with the library's own kernels.

    python -m paper_2210_12252_gb300.train_precond [--train 256] [--heldout 64] [--epochs 8]

Training data: residual / target-correction pairs recorded by hw_solve_eigs_traced from plain
solves (TPA preconditioner) on the random-potential family of the tube geometry
(inputs.tube_family: 20-60 wells, depth 2-6 Ha, width 0.6-1.2 bohr).  Each recorded column
gives (R_j, E_j, theta_j) with E_j = (I - X X^H) X* X*^H x_j the part of the converged
subspace the current block still misses.  The network is trained with hw_mlp_train_step
(forward, loss, backward and Adam all in libhelicwave.so) and evaluated on held-out members by
the iterations LOBPCG needs to reach residual 1e-6, against the TPA diagonal.
Writes the FP32 parameters to precond_weights.npy next to this file and a JSON summary.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "precond_weights.npy")
REC_ITERS = [1, 2, 4, 7, 11, 16, 24]


def init_params(seed=0):
    """He-initialised hidden layers and a zero last layer: the untrained network is TPA."""
    g = np.random.default_rng(seed)
    W1 = g.standard_normal((64, 6)) * np.sqrt(2.0 / 6)
    W2 = g.standard_normal((64, 64)) * np.sqrt(2.0 / 64)
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), np.zeros(64),
                           np.zeros(1)]).astype(np.float32)


def load_weights(path=WEIGHTS):
    return np.load(path).astype(np.float32)


def make_context(device=0):
    import torch
    from . import build, helicwave as hw, inputs
    build.build()
    ctx = hw.Context(device)
    L = int(ctx.setup_basis(inputs.GEOM_TUBE, [0.0])[0])
    return ctx, L


def generate(ctx, L, indices, block, tol=1e-6, prec="mixed"):
    """Traced TPA solves; returns a list of batches (R, E, theta, vdiag) on the device."""
    import torch
    from . import inputs
    batches = []
    iters = []
    for idx in indices:
        w = inputs.tube_family(idx)
        ctx.build_potential(w.atoms)
        vd = torch.from_numpy(ctx.potential_diagonal(0)).cuda()
        r = ctx.solve_traced(0, w.n_eig, block, REC_ITERS, tol=tol, maxit=400, prec=prec)
        if not r["converged"]:
            continue
        iters.append(r["iters"])
        for q, it in enumerate(REC_ITERS):
            if it >= r["iters"]:
                break
            act = np.nonzero(r["res"][q] > 10 * tol)[0]
            if act.size < 4:
                continue
            sel = torch.from_numpy(act).cuda()
            batches.append((r["R"][q].index_select(0, sel).contiguous(),
                            r["E"][q].index_select(0, sel).contiguous(),
                            r["theta"][q][act].copy(), vd))
    return batches, iters


def evaluate(ctx, L, indices, params, block, tol=1e-6, prec="mixed"):
    from . import inputs
    out = []
    for idx in indices:
        w = inputs.tube_family(idx)
        ctx.build_potential(w.atoms)
        row = {"index": int(idx)}
        for pc in ("tpa", "learned"):
            if pc == "learned":
                ctx.set_mlp(params)
            t = time.perf_counter()
            r = ctx.solve_eigs([0], w.n_eig, block=block, tol=tol, maxit=600, prec=prec, precond=pc)
            row[pc] = {"iters": int(r["iters"][0]), "seconds": time.perf_counter() - t,
                       "converged": bool(r["converged"])}
        out.append(row)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=256)
    ap.add_argument("--heldout", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--summary", default=os.path.join(HERE, "precond_training.json"))
    args = ap.parse_args()
    ctx, L = make_context()
    block = 72
    params = init_params(0)
    ctx.set_mlp(params)
    t0 = time.perf_counter()
    batches, it_train = generate(ctx, L, range(args.train), block)
    t_gen = time.perf_counter() - t0
    print(f"{len(batches)} batches from {len(it_train)} solves in {t_gen:.1f} s", file=sys.stderr)
    rng = np.random.default_rng(0)
    hist = []
    t0 = time.perf_counter()
    nsteps = 0
    for ep in range(args.epochs):
        lr = args.lr * (0.5 ** (ep / max(1, args.epochs / 3)))
        order = rng.permutation(len(batches))
        tot = 0.0
        for b in order:
            R, E, th, vd = batches[b]
            tot += ctx.mlp_train_step(0, R, E, th, lr, vdiag=vd)
            nsteps += 1
        hist.append(tot / len(batches))
        print(f"epoch {ep}: mean loss {hist[-1]:.5f} (lr {lr:.2e})", file=sys.stderr)
    t_train = time.perf_counter() - t0
    params = ctx.get_mlp()
    np.save(args.out, params)
    # loss of the untrained (TPA) network on the same data, for reference
    ctx.set_mlp(init_params(0))
    base = np.mean([ctx.mlp_loss_grad(0, R, E, th, vdiag=vd, want_grad=False)[0] for R, E, th, vd in batches])
    ctx.set_mlp(params)
    ev = evaluate(ctx, L, range(256, 256 + args.heldout), params, block)
    it_tpa = np.mean([r["tpa"]["iters"] for r in ev])
    it_ml = np.mean([r["learned"]["iters"] for r in ev])
    summ = {"train_potentials": args.train, "heldout_potentials": args.heldout,
            "batches": len(batches), "train_steps": nsteps, "epochs": args.epochs,
            "loss_tpa": float(base), "loss_per_epoch": [float(x) for x in hist],
            "generate_seconds": t_gen, "train_seconds": t_train,
            "heldout_mean_iters_tpa": float(it_tpa), "heldout_mean_iters_learned": float(it_ml),
            "heldout_mean_seconds_tpa": float(np.mean([r["tpa"]["seconds"] for r in ev])),
            "heldout_mean_seconds_learned": float(np.mean([r["learned"]["seconds"] for r in ev])),
            "heldout": ev}
    with open(args.summary, "w") as f:
        json.dump(summ, f, indent=1)
    print(json.dumps({k: v for k, v in summ.items() if k != "heldout"}))


if __name__ == "__main__":
    main()
