"""Train the L-level network on systems the method itself generates (Sec. 4.2.3).

The paper's training set (107 matrices from 11 simulation scenes, 800
right-hand sides each from 1600 Ritz vectors) is not available; this driver
builds its stand-in on the GPU:

* systems: seeded sloshing scenes (solid shell, 10-40 solid spheres/boxes, a
  sinusoidal free surface) at 64^3 and 128^3, one frame each;
* right-hand sides (--rhs-mode paper, the paper's recipe): per system, m =
  1600 Lanczos steps on A with full reorthogonalisation, and `--rhs` (800)
  random normalised combinations of all the Ritz vectors;
  (--rhs-mode mixed, the earlier reduced recipe): half of them combinations of
  the 32 lowest Ritz vectors of 48 Lanczos steps, half N(0, 1) on the fluid
  cells (projected per pure-Neumann component), all of unit length;
* each step draws a batch of `--per-batch` systems at each size, one
  right-hand side each, and takes one Adam step on the mean of the
  per-system losses || b - A P_net(I, b) ||_2, with the library's
  hand-written backward.  The learning rate falls from `--lr` to a tenth of
  it over the last 40% of each stage's time.

Stages (--stages, e.g. "4:12,5:8,6:10"): each trains an L-level network for
the given minutes.  A stage with one level more than the previous one starts
from the transfer of the previous network (the paper trains a 5-level network
and uses its weights to initialise a 6-level one): the old coarsest level
becomes level L-1 with Aff1 = 1 and Aff2 = 0 there, so the new network
computes exactly the old one before training, and the new level's blocks start
from the seeded initialisation.  "3:8:scratch" starts from the seeded
initialisation instead.  The first stage starts from --init when given.

After each stage the weights are written as raw FP32
(npsolve_weight_count(L) values) to <out-dir>/npsdo_L<L>.f32 with a JSON log
beside them (loss history, the iteration counts of the 256^3 / 128^3 / 64^3
evaluation problems in both precision forms).

--time-steps K times K training steps instead (after one untimed step) on a
fixed batch of 8 seeded 64^3 and 8 seeded 128^3 sloshing systems with N(0, 1)
right-hand sides (the cost of a step does not depend on them) at lr 1e-30, so
that the weights stay as they are; --levels picks the network (its trained
weights when present).
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

CCONV_PARAMS = 27 * 3 * 27 + 27
AFF_PARAMS = 3 * 27 + 1
PER_LEVEL = 2 * CCONV_PARAMS + 2 * AFF_PARAMS


def transfer_weights(w, L, seed=7):
    """The weights of an (L+1)-level network that computes exactly what the
    L-level network `w` computes: levels 1..L-1 unchanged; level L keeps its
    CConv1 and gets Aff1 = 1 (Wbar = 0, Bbar = 1) and Aff2 = 0, so that
    x^L = CConv1^L(r^L) as before; level L's CConv2 and level L+1's CConv1
    come from the seeded initialisation (they enter through Aff2 only)."""
    from paper_2310_00177_b300 import synth

    w = np.asarray(w, np.float64)
    assert w.size == (L - 1) * PER_LEVEL + CCONV_PARAMS
    fresh = synth.init_weights(L + 1, seed)
    out = fresh.copy()
    out[: (L - 1) * PER_LEVEL] = w[: (L - 1) * PER_LEVEL]
    o = (L - 1) * PER_LEVEL
    out[o:o + CCONV_PARAMS] = w[o:o + CCONV_PARAMS]
    a1 = o + 2 * CCONV_PARAMS
    out[a1:a1 + AFF_PARAMS] = 0.0
    out[a1 + AFF_PARAMS - 1] = 1.0
    a2 = a1 + AFF_PARAMS
    out[a2:a2 + AFF_PARAMS] = 0.0
    return out.astype(np.float32)


def make_pool(n, count, rhs_per_system, mode, seed, dev):
    """Systems of size n^3 with their right-hand sides (device tensors)."""
    import torch

    from paper_2310_00177_b300 import binding, synth

    pool = []
    for i in range(count):
        lab = synth.slosh_scene(n, seed + i, frame=(i * 3) % 17)
        labd = torch.from_numpy(lab).to(dev)
        start = torch.from_numpy(synth.rhs_normal(lab, seed * 7 + i).astype(np.float32)).to(dev)
        if mode == "paper":
            combos, _ = binding.lanczos_rhs(labd, start, m=1600, k=1600, count=rhs_per_system, seed=seed * 13 + i)
            rhs = combos
        else:
            n_ritz = rhs_per_system // 2
            rhs = []
            if n_ritz:
                combos, _ = binding.lanczos_rhs(labd, start, m=48, k=32, count=n_ritz, seed=seed * 13 + i)
                rhs += [combos[j] for j in range(n_ritz)]
            for j in range(rhs_per_system - n_ritz):
                b = synth.rhs_normal(lab, seed * 17 + 31 * i + j)
                rhs.append(torch.from_numpy((b / np.linalg.norm(b)).astype(np.float32)).to(dev))
        pool.append((labd, rhs))
        torch.cuda.synchronize()
    return pool


def evaluate(w, L, dev):
    """Iterations (and ms) of the evaluation problems: the benchmark's 256^3
    problem and the 128^3 / 64^3 sloshing problems, both precision forms."""
    import torch

    from paper_2310_00177_b300 import binding, synth

    res = {}
    for n, s_lab, s_rhs in ((256, 3000, 3001), (128, 2000, 2001), (64, 2000, 2001)):
        lab = torch.from_numpy(synth.slosh_scene(n, s_lab)).to(dev)
        rhs = torch.from_numpy(synth.rhs_normal(lab.cpu().numpy(), s_rhs).astype(np.float32)).to(dev)
        for prec, name in ((binding.BF16, "bf16"), (binding.FP32, "fp32")):
            s = binding.Solver(w, levels=L, n_ortho=2, precision=prec)
            s.solve(lab, rhs, 1e-6, 3000)
            torch.cuda.synchronize()
            t = time.perf_counter()
            _, it, rr, st = s.solve(lab, rhs, 1e-6, 3000)
            torch.cuda.synchronize()
            res[f"{n}_{name}"] = {"iters": it, "relres": rr, "status": binding.STATUS_NAMES[st],
                                  "ms": (time.perf_counter() - t) * 1e3}
            s.close()
    return res


def parse_stages(text):
    out = []
    for part in text.split(","):
        f = part.split(":")
        out.append((int(f[0]), float(f[1]), f[2] if len(f) > 2 else "prev"))
    return out


def train_stage(w0, L, minutes, lr0, pools, per_batch, rng, log_every=50):
    from paper_2310_00177_b300 import binding

    sol = binding.Solver(w0, levels=L, n_ortho=2, precision=binding.FP32)
    hist = []
    t1 = time.time()
    step = 0
    budget = minutes * 60
    while time.time() - t1 < budget:
        frac = (time.time() - t1) / budget
        lr = lr0 if frac < 0.6 else lr0 * 10 ** (-(frac - 0.6) / 0.4)
        labs, bs = [], []
        for pool in pools:
            for _ in range(per_batch):
                i = rng.integers(len(pool))
                rh = pool[i][1]
                j = rng.integers(len(rh))
                labs.append(pool[i][0])
                bs.append(rh[j])
        hist.append(sol.train_step(labs, bs, lr=lr))
        step += 1
        if step % log_every == 0:
            print(f"L={L} step {step} loss {np.mean(hist[-log_every:]):.5f} lr {lr:.2e} ({time.time() - t1:.0f} s)",
                  flush=True)
    w = sol.get_weights()
    sol.close()
    return w, hist, time.time() - t1


def time_steps(steps, L, dev):
    """ms per training step on the fixed timing batch (--time-steps)."""
    import torch

    from paper_2310_00177_b300 import binding, synth

    f = os.path.join(ROOT, "paper_2310_00177_b300", "weights", f"npsdo_L{L}.f32")
    w = np.fromfile(f, np.float32) if os.path.exists(f) else synth.init_weights(L, 7).astype(np.float32)
    sol = binding.Solver(w, levels=L, n_ortho=2, precision=binding.FP32)
    labs, bs = [], []
    for i, n in enumerate([64] * 8 + [128] * 8):
        lab = synth.slosh_scene(n, 5000 + i)
        b = synth.rhs_normal(lab, 6000 + i).astype(np.float32)
        b /= max(float(np.linalg.norm(b)), 1e-30)
        labs.append(torch.from_numpy(lab).to(dev))
        bs.append(torch.from_numpy(b).to(dev))
    sol.train_step(labs, bs, lr=1e-30)
    out = []
    for _ in range(steps):
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        loss = sol.train_step(labs, bs, lr=1e-30)
        torch.cuda.synchronize(dev)
        out.append((time.perf_counter() - t) * 1e3)
    sol.close()
    print(json.dumps({"levels": L, "batch": "8 x 64^3 + 8 x 128^3", "ms_per_step": out, "loss": loss}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--stages", default="4:8", help="comma-separated L:minutes[:scratch]")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--systems", type=int, default=12, help="systems per size")
    ap.add_argument("--rhs", type=int, default=800, help="right-hand sides per system")
    ap.add_argument("--rhs-mode", default="paper", choices=["paper", "mixed"])
    ap.add_argument("--small", type=int, default=64)
    ap.add_argument("--large", type=int, default=128)
    ap.add_argument("--per-batch", type=int, default=8, help="systems of each size per step")
    ap.add_argument("--init", default="", help="initial weights of the first stage (default: seeded init)")
    ap.add_argument("--out-dir", default=os.path.join(ROOT, "paper_2310_00177_b300", "weights"))
    ap.add_argument("--seed", type=int, default=4000)
    ap.add_argument("--no-eval", action="store_true")
    ap.add_argument("--time-steps", type=int, default=0, help="only time this many steps on the timing batch")
    ap.add_argument("--levels", type=int, default=6, help="network depth of --time-steps")
    args = ap.parse_args()

    import torch

    from paper_2310_00177_b300 import synth

    dev = torch.device("cuda", 0)
    if args.time_steps:
        time_steps(args.time_steps, args.levels, dev)
        return
    t0 = time.time()
    pool_s = make_pool(args.small, args.systems, args.rhs, args.rhs_mode, args.seed, dev)
    t_s = time.time() - t0
    pool_l = make_pool(args.large, args.systems, args.rhs, args.rhs_mode, args.seed + 1000, dev)
    t_gen = time.time() - t0
    print(f"right-hand sides: {t_s:.0f} s at {args.small}^3, {t_gen - t_s:.0f} s at {args.large}^3", flush=True)
    rng = np.random.default_rng(args.seed)
    os.makedirs(args.out_dir, exist_ok=True)
    w, L_prev = None, None
    for si, (L, minutes, src) in enumerate(parse_stages(args.stages)):
        if src == "scratch" or (w is None and not args.init):
            w0, how = synth.init_weights(L, 7).astype(np.float32), "seeded init"
        elif w is None:
            w0 = np.fromfile(args.init, dtype=np.float32)
            L_init = next(l for l in range(1, 8) if (l - 1) * PER_LEVEL + CCONV_PARAMS == w0.size)
            how = f"{os.path.basename(args.init)} (L={L_init})"
            while L_init < L:
                w0 = transfer_weights(w0, L_init)
                L_init += 1
                how += f" -> transfer to L={L_init}"
        elif L == L_prev:
            w0, how = w, "previous stage"
        elif L == L_prev + 1:
            w0, how = transfer_weights(w, L_prev), f"transfer from the L={L_prev} stage"
        else:
            raise SystemExit(f"stage {si}: L={L} does not follow L={L_prev}")
        wl, hist, secs = train_stage(w0, L, minutes, args.lr, (pool_s, pool_l), args.per_batch, rng)
        out = os.path.join(args.out_dir, f"npsdo_L{L}.f32")
        wl.astype(np.float32).tofile(out)
        log = {"levels": L, "start": how, "steps": len(hist), "seconds": secs, "lr": args.lr,
               "rhs_mode": args.rhs_mode, "systems_per_size": args.systems, "rhs_per_system": args.rhs,
               "sizes": [args.small, args.large], "per_batch": args.per_batch,
               "rhs_generation_seconds": t_gen, "loss_first": hist[0] if hist else None,
               "loss_last50": float(np.mean(hist[-50:])) if hist else None,
               "loss_history": [float(v) for v in hist[::max(1, len(hist) // 200)]]}
        if not args.no_eval:
            log["evaluation"] = evaluate(wl, L, dev)
        json.dump(log, open(os.path.splitext(out)[0] + "_train.json", "w"), indent=1)
        print(json.dumps({k: v for k, v in log.items() if k != "loss_history"}), flush=True)
        w, L_prev = wl, L


if __name__ == "__main__":
    main()
