"""Store the FP64 oracle's own solve of a benchmark problem.

TEST INFRASTRUCTURE: calls only the CPU oracle (and the seeded input
generators).  The full-size parity tests compare the CUDA library's solves
with what this script stores, since an oracle solve at 256^3 takes about half
an hour on the host cores; the benchmark's reference arm scales its
per-iteration time by the stored iteration count.

The problems are the sloshing scenes of the benchmark: 256^3 (scene seed
3000, right-hand side seed 3001) and 128^3 (scene seed 2000, right-hand side
seed 2001), L levels (--levels, default 4) with the network weights
paper_2310_00177_b300/weights/npsdo_L<L>.f32 identified by their SHA-256,
n_ortho = 2, tol 1e-6, recurrence residual.  --form bf16 solves with the
oracle's model of the library's BF16 form (every CConv kernel value rounded
to BF16) instead of the exact FP64 network.

Stored: the iteration count, the status, the relative residual history and a
compact record of x.  x is unique only up to a constant on each fluid
component that touches no air (the matrix is singular there), so the record
holds x with each such component's mean removed: its values at 4096 seeded
fluid cells, the sum and the 2-norm of every z-plane, and its 2-norm.

Usage: python oracle/count_iterations.py [--n 256] [--form fp64|bf16] [--levels 4]
                                         [--weights FILE] [--out FILE]
"""
import argparse
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2310_00177_b300 import synth  # noqa: E402

SEEDS = {256: (3000, 3001), 128: (2000, 2001)}
N_SAMPLES = 4096


def weights_id(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def default_out(n, form, levels=4):
    return os.path.join(HERE, f"iterations_slosh{n}" + ("_bf16" if form == "bf16" else "") +
                        (f"_L{levels}" if levels != 4 else "") + ".json")


def remove_neumann_constants(labels, x):
    """x with its mean removed on every pure-Neumann fluid component."""
    comp, pure = synth.neumann_components(labels)
    x = x.copy()
    for c in pure:
        m = comp == c
        x[m] -= x[m].mean()
    return x


def sample_cells(labels, count=N_SAMPLES, seed=12345):
    """Flat indices of `count` seeded fluid cells, sorted."""
    fluid = np.flatnonzero(labels.ravel() == 1)
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(fluid, size=min(count, fluid.size), replace=False))


def x_record(labels, x):
    xc = remove_neumann_constants(labels, x)
    cells = sample_cells(labels)
    return {"cells": [int(c) for c in cells], "values": [float(v) for v in xc.ravel()[cells]],
            "plane_sum": [float(v) for v in xc.sum(axis=(1, 2))],
            "plane_norm": [float(v) for v in np.sqrt((xc * xc).sum(axis=(1, 2)))],
            "norm": float(np.linalg.norm(xc))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256, choices=sorted(SEEDS))
    ap.add_argument("--form", default="fp64", choices=["fp64", "bf16"])
    ap.add_argument("--levels", type=int, default=4)
    ap.add_argument("--weights", default=None, help="default: paper_2310_00177_b300/weights/npsdo_L<levels>.f32")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    if args.weights is None:
        args.weights = os.path.join(ROOT, "paper_2310_00177_b300", "weights", f"npsdo_L{args.levels}.f32")
    out_path = args.out or default_out(args.n, args.form, args.levels)
    s_lab, s_rhs = SEEDS[args.n]
    lab = synth.slosh_scene(args.n, s_lab)
    rhs = synth.rhs_normal(lab, s_rhs).astype(np.float32)
    w = np.fromfile(args.weights, dtype=np.float32)
    prec = oracle.PREC_NETWORK_BF16 if args.form == "bf16" else oracle.PREC_NETWORK
    t = time.time()
    res = oracle.npsdo(lab, rhs.astype(np.float64), L=args.levels, w=w.astype(np.float64), tol=1e-6, max_iter=2000,
                       prec=prec)
    out = {"n": args.n, "form": args.form, "levels": args.levels, "scene_seed": s_lab, "rhs_seed": s_rhs,
           "weights_sha256_16": weights_id(args.weights), "iters": res["iters"], "status": res["status"],
           "relres": res["relres"], "seconds": time.time() - t,
           "res_hist": [float(v) for v in res["res_hist"] / res["res_hist"][0]],
           "x_record": x_record(lab, res["x"])}
    json.dump(out, open(out_path, "w"), indent=0)
    print(json.dumps({k: v for k, v in out.items() if k not in ("res_hist", "x_record")}))


if __name__ == "__main__":
    main()
