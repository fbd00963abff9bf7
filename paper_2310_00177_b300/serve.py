"""Serving driver: a stream of solve requests through the continuous-batching
server (npsolve_server_*), reporting p50 / p99 latency and solves per second.

The request stream follows the deployment setting: Poisson arrivals (mean
rate `rate` per second), grid sizes drawn uniformly from `sizes`, each request
a frame of an evolving scene of its size (solids translating one cell per
frame along x, the free surface sloshing), b ~ N(0, 1) on the fluid cells,
BF16 network, tolerance 1e-6, admission by an HBM budget.  Frames are
generated up front (`frames` distinct frames per size, reused cyclically) so
that generation does not perturb the arrival clock.

Latency of a request = time from its nominal arrival to the end of its solve
(including the copy of x back to the host), measured inside the server plus
the driver's lag in submitting; throughput = completed solves / (last
completion - first arrival).
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


def build_frames(sizes, frames, seed=5000, pinned=False):
    from paper_2310_00177_b300 import synth

    out = {}
    for n in sizes:
        lst = []
        for f in range(frames):
            lab = synth.slosh_scene(n, seed + n, frame=f)
            b = synth.rhs_normal(lab, seed * 3 + 101 * n + f).astype(np.float32)
            if pinned:
                lp, bp = pinned_like(lab.shape, np.uint8), pinned_like(b.shape, np.float32)
                lp[...] = lab
                bp[...] = b
                lab, b = lp, bp
            lst.append((lab, b))
        out[n] = lst
    return out


def run(server, requests, frames, tol=1e-6, max_iter=2000, keep_x=None, x_pool=None):
    """Submit `requests` (dicts with t_arrival, n, frame) at their arrival times
    and collect the results.  x of request i goes to x_pool[i] when given
    (pinned host arrays), else to a fresh array for the indices in keep_x,
    else is not copied back.  Latency = end of the solve - nominal arrival."""
    t0 = time.perf_counter()
    recs = {}
    pending = set()
    keep_x = keep_x or set()
    i = 0

    def drain():
        for rid in server.poll():
            meta = recs[rid]
            x, it, rr, st, qms, sms = server.result(rid)
            meta.update(iters=it, relres=rr, status=st, queue_ms=qms, service_ms=sms)
            # the server times submit -> end; add the driver's lag behind the nominal arrival
            meta["latency_ms"] = meta["submit_lag_ms"] + qms + sms
            meta["t_done"] = meta["t_arrival"] + meta["latency_ms"] / 1e3
            if x is not None and meta["index"] in keep_x:
                meta["x"] = x.copy()
            pending.discard(rid)

    while i < len(requests) or pending:
        now = time.perf_counter() - t0
        while i < len(requests) and requests[i]["t_arrival"] <= now:
            req = requests[i]
            lab, b = frames[req["n"]][req["frame"] % len(frames[req["n"]])]
            if x_pool is not None:
                x = x_pool[i]
            elif i in keep_x:
                x = np.empty(lab.shape, np.float64)
            else:
                x = None
            lag = (time.perf_counter() - t0 - req["t_arrival"]) * 1e3
            rid = server.submit(lab, b, x=x, tol=tol, max_iter=max_iter)
            recs[rid] = {"index": i, "n": req["n"], "frame": req["frame"], "t_arrival": req["t_arrival"],
                         "shape": lab.shape, "submit_lag_ms": lag}
            pending.add(rid)
            i += 1
        drain()
        if pending or i < len(requests):
            nxt = requests[i]["t_arrival"] - (time.perf_counter() - t0) if i < len(requests) else 0.0005
            time.sleep(max(0.0002, min(nxt, 0.002)))
    return recs


def pinned_like(shape, dtype):
    """A page-locked host array (via torch) for fast copies."""
    import torch

    t = torch.empty(shape, dtype={np.uint8: torch.uint8, np.float32: torch.float32,
                                  np.float64: torch.float64}[np.dtype(dtype).type]).pin_memory()
    return t.numpy()


def summarize(recs):
    lat = np.array([r["latency_ms"] for r in recs.values()])
    t_first = min(r["t_arrival"] for r in recs.values())
    t_last = max(r["t_done"] for r in recs.values())
    by_size = {}
    for r in recs.values():
        by_size.setdefault(r["n"], []).append(r)
    return {
        "requests": len(recs),
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()), "solves_per_s": len(recs) / max(t_last - t_first, 1e-9),
        "all_converged": all(r["status"] == 0 and r["relres"] < 1e-6 for r in recs.values()),
        "per_size": {str(n): {"count": len(v), "iters_mean": float(np.mean([r["iters"] for r in v])),
                              "service_ms_mean": float(np.mean([r["service_ms"] for r in v])),
                              "p50_ms": float(np.percentile([r["latency_ms"] for r in v], 50))}
                     for n, v in sorted(by_size.items())},
    }


def serve_workload(w, requests=512, rate=200.0, sizes=(64, 128, 192, 256), frames=6, budget_gb=150.0,
                   max_active=8, levels=4):
    """Run the serving workload (seeded Poisson arrivals, mixed sizes, evolving
    frames, BF16 network, tol 1e-6, HBM-budget admission) on a fresh server
    and return the summary: p50 / p99 latency, solves per second, convergence
    of every request, peak reserved HBM."""
    from paper_2310_00177_b300 import binding, synth

    sizes = tuple(sizes)
    fr = build_frames(sizes, frames, pinned=True)
    reqs = synth.serving_requests(requests, rate, sizes=sizes)
    # every request returns its x to the host (a pinned array per request)
    x_pool = [pinned_like((r["n"],) * 3, np.float64) for r in reqs]
    srv = binding.Server(w, levels=levels, precision=binding.BF16, hbm_budget_bytes=int(budget_gb * (1 << 30)),
                         max_active=max_active)
    try:
        # grow every slot to the largest size once so that workspace growth is not timed
        warm = run(srv, [{"t_arrival": 0.0, "n": max(sizes), "frame": 0} for _ in range(max_active)], fr)
        recs = run(srv, reqs, fr, x_pool=x_pool)
        out = summarize(recs)
        out["peak_reserved_gb"] = srv.stats()["peak_reserved"] / (1 << 30)
    finally:
        srv.close()
    out["rate_per_s"] = rate
    out["sizes"] = list(sizes)
    out["budget_gb"] = budget_gb
    out["max_active"] = max_active
    out["levels"] = levels
    out["warmup_requests"] = len(warm)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=512)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--sizes", default="64,128,192,256")
    ap.add_argument("--frames", type=int, default=6)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--max-active", type=int, default=8)
    ap.add_argument("--levels", type=int, default=6)
    args = ap.parse_args()
    from paper_2310_00177_b300 import synth

    wfile = os.path.join(ROOT, "paper_2310_00177_b300", "weights", f"npsdo_L{args.levels}.f32")
    w = np.fromfile(wfile, dtype=np.float32) if os.path.exists(wfile) else synth.init_weights(args.levels, 7)
    out = serve_workload(w, args.requests, args.rate, tuple(int(s) for s in args.sizes.split(",")), args.frames,
                         args.budget_gb, args.max_active, args.levels)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
