"""Train the L-level network on systems the method itself generates (Sec. 4.2.3).

The paper's training set (107 matrices from 11 simulation scenes, 800
right-hand sides each from 1600 Ritz vectors) is not available; this driver
builds its stand-in on the GPU:

* systems: seeded sloshing scenes (solid shell, 10-40 solid spheres/boxes, a
  sinusoidal free surface) at 64^3 and 128^3, several frames each;
* right-hand sides: half are random normalised combinations of the lowest
  Ritz vectors of A from a Lanczos run with full reorthogonalisation (the
  paper's recipe at a reduced count), half are N(0, 1) on the fluid cells
  (projected per pure-Neumann component), all normalised to unit length;
* each step draws a batch of 8 systems at 64^3 and 8 at 128^3 and takes one
  Adam step (lr 1e-3) on the mean of the per-system losses
  || b - A P_net(I, b) ||_2, with the library's hand-written backward.

The weights are written as raw FP32 (npsolve_weight_count(L) values) and a
JSON log of the loss history next to them.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402


def make_pool(n, count, rhs_per_system, ritz_k, lanczos_m, seed, dev):
    import torch

    from paper_2310_00177_b300 import binding, synth

    pool = []
    for i in range(count):
        lab = synth.slosh_scene(n, seed + i, frame=(i * 3) % 17)
        labd = torch.from_numpy(lab).to(dev)
        rhs = []
        start = synth.rhs_normal(lab, seed * 7 + i).astype(np.float32)
        n_ritz = rhs_per_system // 2
        if n_ritz:
            combos, _ = binding.lanczos_rhs(labd, torch.from_numpy(start).to(dev), m=lanczos_m, k=ritz_k,
                                            count=n_ritz, seed=seed * 13 + i)
            rhs += [combos[j].contiguous() for j in range(n_ritz)]
        for j in range(rhs_per_system - n_ritz):
            b = synth.rhs_normal(lab, seed * 17 + 31 * i + j)
            b = (b / np.linalg.norm(b)).astype(np.float32)
            rhs.append(torch.from_numpy(b).to(dev))
        pool.append((labd, rhs))
    return pool


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--levels", type=int, default=4)
    ap.add_argument("--minutes", type=float, default=8.0, help="wall-clock training budget")
    ap.add_argument("--max-steps", type=int, default=100000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--systems", type=int, default=12, help="systems per size")
    ap.add_argument("--rhs", type=int, default=8, help="right-hand sides per system")
    ap.add_argument("--small", type=int, default=64)
    ap.add_argument("--large", type=int, default=128)
    ap.add_argument("--per-batch", type=int, default=8, help="systems of each size per step")
    ap.add_argument("--init", default="", help="initial weights file (default: seeded init)")
    ap.add_argument("--out", default=os.path.join(ROOT, "paper_2310_00177_b300", "weights", "npsdo_L4.f32"))
    ap.add_argument("--seed", type=int, default=4000)
    args = ap.parse_args()

    import torch

    from paper_2310_00177_b300 import binding, synth

    dev = torch.device("cuda", 0)
    t0 = time.time()
    pool_s = make_pool(args.small, args.systems, args.rhs, 32, 48, args.seed, dev)
    pool_l = make_pool(args.large, args.systems, args.rhs, 32, 48, args.seed + 1000, dev)
    t_gen = time.time() - t0
    w0 = (np.fromfile(args.init, dtype=np.float32) if args.init
          else synth.init_weights(args.levels, 7).astype(np.float32))
    sol = binding.Solver(w0, levels=args.levels, n_ortho=2, precision=binding.FP32)
    rng = np.random.default_rng(args.seed)
    hist = []
    t1 = time.time()
    step = 0
    while step < args.max_steps and time.time() - t1 < args.minutes * 60:
        labs, bs = [], []
        for pool in (pool_s, pool_l):
            for _ in range(args.per_batch):
                i = rng.integers(len(pool))
                j = rng.integers(len(pool[i][1]))
                labs.append(pool[i][0])
                bs.append(pool[i][1][j])
        lr = args.lr if step < 0.7 * args.max_steps else args.lr * 0.3
        loss = sol.train_step(labs, bs, lr=lr)
        hist.append(loss)
        step += 1
        if step % 25 == 0:
            print(f"step {step} loss {np.mean(hist[-25:]):.5f} ({time.time() - t1:.0f} s)", flush=True)
    w = sol.get_weights()
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    w.astype(np.float32).tofile(args.out)
    log = {"steps": step, "seconds": time.time() - t1, "rhs_generation_seconds": t_gen, "lr": args.lr,
           "levels": args.levels, "systems_per_size": args.systems, "rhs_per_system": args.rhs,
           "sizes": [args.small, args.large], "per_batch": args.per_batch,
           "loss_first": hist[0] if hist else None, "loss_last25": float(np.mean(hist[-25:])) if hist else None,
           "loss_history": hist[::max(1, len(hist) // 200)]}
    json.dump(log, open(os.path.splitext(args.out)[0] + "_train.json", "w"), indent=1)
    print(json.dumps({k: v for k, v in log.items() if k != "loss_history"}))


if __name__ == "__main__":
    main()
