"""Solve one seeded synthetic scene with the library and print what happened.

    python -m paper_2310_00177_b300.solve_scene --n 256 --solves 2

Builds the sloshing scene of the given size (Sec. 5 stand-in: solid shell,
solid spheres and boxes, a sinusoidal free surface), a normal right-hand side
projected per pure-Neumann component, loads the trained weights of the
chosen depth (--levels, default 6, the paper's; a seeded initialisation when
the file is absent) and runs NPSDO (Alg. 1) with
the network preconditioner (Alg. 2).  Prints one JSON line per solve with the
iteration count, the FP64 true relative residual and the wall time.  Useful as
a minimal example of the Python binding and as a fixed command to profile.
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


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128, help="grid size (n^3, divisible by 8)")
    ap.add_argument("--scene-seed", type=int, default=3000)
    ap.add_argument("--rhs-seed", type=int, default=3001)
    ap.add_argument("--solves", type=int, default=1)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-iter", type=int, default=2000)
    ap.add_argument("--precision", choices=["bf16", "fp32"], default="bf16")
    ap.add_argument("--path", choices=["cached", "cuda_core", "tensor"], default="cached")
    ap.add_argument("--levels", type=int, default=6)
    args = ap.parse_args(argv)

    import torch

    from paper_2310_00177_b300 import binding, synth

    wfile = os.path.join(ROOT, "paper_2310_00177_b300", "weights", f"npsdo_L{args.levels}.f32")
    w = (np.fromfile(wfile, dtype=np.float32) if os.path.exists(wfile)
         else synth.init_weights(args.levels, 7).astype(np.float32))
    lab = synth.slosh_scene(args.n, args.scene_seed)
    rhs = synth.rhs_normal(lab, args.rhs_seed).astype(np.float32)
    dev = torch.device("cuda", 0)
    lab_d = torch.from_numpy(lab).to(dev)
    b_d = torch.from_numpy(rhs).to(dev)
    path = {"cached": binding.PATH_CACHED, "cuda_core": binding.PATH_CUDA_CORE, "tensor": binding.PATH_TENSOR}
    sol = binding.Solver(w, levels=args.levels, precision=binding.BF16 if args.precision == "bf16" else binding.FP32,
                         kernel_path=path[args.path])
    for i in range(args.solves):
        torch.cuda.synchronize()
        t = time.perf_counter()
        x, iters, relres, status = sol.solve(lab_d, b_d, args.tol, args.max_iter)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t) * 1e3
        print(json.dumps({"solve": i, "n": args.n, "iters": iters, "relres": relres, "status": status,
                          "ms": round(ms, 3)}), flush=True)
    sol.close()


if __name__ == "__main__":
    main()
