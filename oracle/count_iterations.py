"""Store the FP64 oracle's own NPSDO iteration count for the benchmark problem.

TEST INFRASTRUCTURE: calls only the CPU oracle.  The benchmark's reference arm
(the oracle, timed per iteration on the host cores) scales its per-iteration
time by this count to report milliseconds per solve.  The problem is the
benchmark's 256^3 sloshing scene (scene seed 3000, right-hand side seed 3001),
L = 4, n_ortho = 2, tol 1e-6, recurrence residual, with the network weights
identified by their SHA-256.

Usage: python oracle/count_iterations.py [--n 256] [--weights FILE]
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


def weights_id(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--weights", default=os.path.join(ROOT, "paper_2310_00177_b300", "weights", "npsdo_L4.f32"))
    ap.add_argument("--out", default=os.path.join(HERE, "iterations_slosh256.json"))
    args = ap.parse_args()
    lab = synth.slosh_scene(args.n, 3000)
    rhs = synth.rhs_normal(lab, 3001).astype(np.float32)
    w = np.fromfile(args.weights, dtype=np.float32)
    t = time.time()
    res = oracle.npsdo(lab, rhs.astype(np.float64), L=4, w=w.astype(np.float64), tol=1e-6, max_iter=2000)
    out = {"n": args.n, "weights_sha256_16": weights_id(args.weights), "iters": res["iters"],
           "status": res["status"], "relres": res["relres"], "seconds": time.time() - t,
           "res_hist": [float(v) for v in res["res_hist"] / res["res_hist"][0]]}
    json.dump(out, open(args.out, "w"), indent=1)
    print(json.dumps({k: v for k, v in out.items() if k != "res_hist"}))


if __name__ == "__main__":
    main()
