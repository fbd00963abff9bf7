"""The continuous-batching server: results identical alone and in the mix,
admission within the HBM budget, every request converged.

Identity: every slot runs the same deterministic kernels (fixed reduction
orders, no atomics in any value path), so a request solved among others must
give bit-for-bit the x and the iteration count of the same request solved on
its own handle."""
import numpy as np
import pytest

from paper_2310_00177_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _b():
    from paper_2310_00177_b300 import binding

    return binding


def _weights():
    import os

    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    f = os.path.join(here, "paper_2310_00177_b300", "weights", "npsdo_L4.f32")
    return np.fromfile(f, dtype=np.float32) if os.path.exists(f) else synth.init_weights(4, 7).astype(np.float32)


def test_results_identical_alone_and_in_the_mix():
    b = _b()
    from paper_2310_00177_b300 import serve

    w = _weights()
    sizes = (32, 48, 64)
    frames = serve.build_frames(sizes, 3, seed=77)
    reqs = [{"t_arrival": 0.002 * i, "n": sizes[i % 3], "frame": i // 3} for i in range(12)]
    srv = b.Server(w, precision=b.BF16, max_active=4)
    recs = serve.run(srv, reqs, frames, keep_x=set(range(12)))
    assert len(recs) == 12
    srv.close()
    alone = b.Solver(w, precision=b.BF16)
    for rid, r in recs.items():
        lab, rhs = frames[r["n"]][r["frame"] % 3]
        x, it, rr, st = alone.solve(torch.from_numpy(lab).cuda(), torch.from_numpy(rhs).cuda(), 1e-6, 2000)
        assert r["status"] == 0 and st == 0
        assert r["iters"] == it
        assert r["relres"] == rr
        np.testing.assert_array_equal(r["x"], x.cpu().numpy())
    alone.close()


def test_admission_respects_the_hbm_budget():
    b = _b()
    from paper_2310_00177_b300 import serve

    w = _weights()
    frames = serve.build_frames((64,), 2, seed=78)
    est = 256 * 64 ** 3 + (64 << 20)  # the server's upper estimate for one 64^3 solve
    budget = int(2.5 * est)            # room for two concurrent 64^3 solves
    srv = b.Server(w, precision=b.BF16, hbm_budget_bytes=budget, max_active=6)
    reqs = [{"t_arrival": 0.0, "n": 64, "frame": i} for i in range(6)]
    recs = serve.run(srv, reqs, frames)
    st = srv.stats()
    srv.close()
    assert len(recs) == 6 and all(r["status"] == 0 and r["relres"] < 1e-6 for r in recs.values())
    assert 0 < st["peak_reserved"] <= budget
    # a request that cannot fit the budget at all is refused
    small = b.Server(w, precision=b.BF16, hbm_budget_bytes=1 << 20, max_active=1)
    with pytest.raises(b.NpsolveError):
        small.submit(frames[64][0][0], frames[64][0][1])
    small.close()


def test_slot_regrowth_at_the_served_sizes():
    # One slot, so every request lands on it: a 64^3 request, then a 256^3
    # one (the handle's workspace and staging buffers grow), then the same two
    # without x (the slot's own request buffers are freed and reallocated
    # larger).  Each result must equal the same request solved alone.
    b = _b()
    from paper_2310_00177_b300 import serve

    w = _weights()
    frames = serve.build_frames((64, 256), 1, seed=79)
    srv = b.Server(w, precision=b.BF16, max_active=1)
    order = [(64, True), (256, True), (64, False), (256, False)]
    xs, ids = {}, []
    for n, keep in order:
        lab, rhs = frames[n][0]
        x = np.empty(lab.shape, np.float64) if keep else None
        ids.append(srv.submit(lab, rhs, x=x, tol=1e-6, max_iter=2000))
        xs[ids[-1]] = x
    done = {}
    import time

    t0 = time.time()
    while len(done) < len(ids) and time.time() - t0 < 120:
        for rid in srv.poll():
            done[rid] = srv.result(rid)
        time.sleep(0.005)
    srv.close()
    assert len(done) == len(ids)
    alone = b.Solver(w, precision=b.BF16)
    ref = {}
    for n in (64, 256):
        lab, rhs = frames[n][0]
        x, it, rr, st = alone.solve(torch.from_numpy(lab).cuda(), torch.from_numpy(rhs).cuda(), 1e-6, 2000)
        assert st == b.OK
        ref[n] = (x.cpu().numpy(), it, rr)
    alone.close()
    for rid, (n, keep) in zip(ids, order):
        x, it, rr, st, _, _ = done[rid]
        assert st == b.OK and it == ref[n][1] and rr == ref[n][2], (n, keep)
        if keep:
            np.testing.assert_array_equal(x, ref[n][0])


def test_result_before_poll_releases_the_request():
    # npsolve_server_result may be called for a finished request that no poll
    # has returned yet; the request is released and no later poll reports it
    b = _b()
    from paper_2310_00177_b300 import serve
    import time

    w = _weights()
    frames = serve.build_frames((32,), 1, seed=80)
    srv = b.Server(w, precision=b.BF16, max_active=2)
    lab, rhs = frames[32][0]
    rid = srv.submit(lab, rhs, x=np.empty(lab.shape, np.float64))
    t0 = time.time()
    while True:  # wait through the stats call, not the poll
        s = srv.stats()
        if s["active"] == 0 and s["queued"] == 0:
            break
        assert time.time() - t0 < 60
        time.sleep(0.002)
    x, it, rr, st, _, _ = srv.result(rid)
    assert st == b.OK and rr < 1e-6 and it > 0
    assert srv.poll() == []
    with pytest.raises(b.NpsolveError):
        srv.result(rid)
    srv.close()
