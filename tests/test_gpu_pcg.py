"""PCG and flexible PCG with the network as preconditioner (Sec. 4.1; the
appendix's comparison of solver variants): the CUDA path (through the C ABI,
npsolve_config.method) against the FP64 oracle's ``npcg``.

Tolerances as for NPSDO (FP32 form): the iteration count matches when the
oracle's last two residuals are at least 5% away from tol*||b|| (else within
one), ||x - x_oracle|| / ||x_oracle|| <= 2e-5 after removing the constants of
pure-Neumann components.  The GPU forms beta with r_k - r_{k-1} = -alpha_k A d_k
(flexible PCG) and the directions scaled by 1/||r_k|| (both exact in exact
arithmetic), so agreement is to FP32 rounding, not bitwise.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2310_00177_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))


def _b():
    from paper_2310_00177_b300 import binding

    return binding


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _nc(labels, x):
    comp, pure = synth.neumann_components(labels)
    x = x.copy()
    for c in pure:
        m = comp == c
        x[m] -= x[m].mean()
    return x


def _trained():
    return np.fromfile(os.path.join(HERE, "..", "paper_2310_00177_b300", "weights", "npsdo_L4.f32"), np.float32)


def _check_count(iters, ores, tol):
    h = ores["res_hist"] / ores["res_hist"][0]
    if h[-1] < 0.95 * tol and h[-2] > 1.05 * tol:
        assert iters == ores["iters"]
    else:
        assert abs(iters - ores["iters"]) <= 1


@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("scene,kernel_path,mode", [
    ("pool32", 0, 0),   # cached kernels, fused CConv2 dots, residual update fused into the next CConv1
    ("pool32", 1, 0),   # CUDA-core kernels: the vectorised combination computes the dots
    ("slosh32", 0, 1),  # explicit residual (one residual buffer)
    ("slosh64", 0, 0),
])
def test_solve_matches_oracle(method, scene, kernel_path, mode):
    b = _b()
    lab = synth.pool_scene(32, 1000) if scene == "pool32" else synth.slosh_scene(int(scene[5:]), 77)
    rhs = synth.rhs_normal(lab, 1001).astype(np.float32)
    w = _trained()
    ores = oracle.npcg(lab, rhs.astype(np.float64), L=4, w=w.astype(np.float64), tol=1e-6, max_iter=500,
                       flexible=method == 2, residual_mode=mode)
    assert ores["status"] == oracle.OK
    s = b.Solver(w, levels=4, method=method, kernel_path=kernel_path, residual_mode=mode)
    x, iters, relres, st = s.solve(_dev(lab, torch.uint8), _dev(rhs, torch.float32), tol=1e-6, max_iter=500)
    assert st == b.OK and relres < 1e-6
    _check_count(iters, ores, 1e-6)
    assert _rel(_nc(lab, x.cpu().numpy()), _nc(lab, ores["x"])) <= 2e-5
    hist = s.residual_history()
    m = min(len(hist), len(ores["res_hist"]))
    np.testing.assert_allclose(hist[:m] / hist[0], ores["res_hist"][:m] / ores["res_hist"][0], rtol=1e-3, atol=1e-9)
    s.close()


@pytest.mark.parametrize("method", [1, 2])
def test_truncated_x_matches_oracle(method):
    # x after a fixed number of iterations; the ring of two directions adds two
    # steps to x at a time in the recurrence mode, so odd and even counts differ
    b = _b()
    lab = synth.slosh_scene(32, 81)
    rhs = synth.rhs_normal(lab, 82).astype(np.float32)
    w = synth.init_weights(4, 83).astype(np.float32)
    s = b.Solver(w, levels=4, method=method)
    for m in range(1, 5):
        ores = oracle.npcg(lab, rhs.astype(np.float64), L=4, w=w.astype(np.float64), tol=1e-12, max_iter=m,
                           flexible=method == 2)
        x, iters, relres, st = s.solve(_dev(lab, torch.uint8), _dev(rhs, torch.float32), tol=1e-12, max_iter=m)
        assert st == b.NO_CONVERGENCE and iters == ores["iters"] == m
        assert _rel(_nc(lab, x.cpu().numpy()), _nc(lab, ores["x"])) <= 2e-5
    s.close()


@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("shape,L", [((6, 10, 14), 2), ((9, 7, 11), 1)])
def test_generic_path_truncated_matches_oracle(method, shape, L):
    # nx % 4 != 0: the general kernels (the dots in the plain combination kernel)
    b = _b()
    lab = np.random.default_rng(41).choice(np.array([0, 1, 2], np.uint8), size=shape, p=(0.15, 0.7, 0.15))
    rhs = synth.rhs_normal(lab, 42).astype(np.float32)
    w = synth.init_weights(L, 43).astype(np.float32)
    s = b.Solver(w, levels=L, method=method)
    for m in (1, 2, 7):
        ores = oracle.npcg(lab, rhs.astype(np.float64), L=L, w=w.astype(np.float64), tol=1e-12, max_iter=m,
                           flexible=method == 2)
        x, iters, relres, st = s.solve(_dev(lab, torch.uint8), _dev(rhs, torch.float32), tol=1e-12, max_iter=m)
        assert st == b.NO_CONVERGENCE and iters == m
        assert _rel(_nc(lab, x.cpu().numpy()), _nc(lab, ores["x"])) <= 2e-5
    s.close()


def test_flexible_pcg_converges_where_oracle_does_on_generic_path():
    b = _b()
    lab = np.random.default_rng(41).choice(np.array([0, 1, 2], np.uint8), size=(6, 10, 14), p=(0.15, 0.7, 0.15))
    rhs = synth.rhs_normal(lab, 42).astype(np.float32)
    w = synth.init_weights(2, 43).astype(np.float32)
    ores = oracle.npcg(lab, rhs.astype(np.float64), L=2, w=w.astype(np.float64), tol=1e-6, max_iter=2000,
                       flexible=True)
    s = b.Solver(w, levels=2, method=b.FPCG)
    x, iters, relres, st = s.solve(_dev(lab, torch.uint8), _dev(rhs, torch.float32), tol=1e-6, max_iter=2000)
    assert st == b.OK and relres < 1e-6
    _check_count(iters, ores, 1e-6)
    s.close()


@pytest.mark.parametrize("method", [1, 2])
def test_bf16_form_converges(method):
    b = _b()
    lab = synth.slosh_scene(64, 4242)
    rhs = synth.rhs_normal(lab, 4243).astype(np.float32)
    w = _trained()
    it = {}
    for prec in (b.FP32, b.BF16):
        s = b.Solver(w, levels=4, method=method, precision=prec)
        _, it[prec], relres, st = s.solve(_dev(lab, torch.uint8), _dev(rhs, torch.float32), tol=1e-6, max_iter=500)
        assert st == b.OK and relres < 1e-6
        s.close()
    assert abs(it[b.BF16] - it[b.FP32]) <= 2


def test_zero_network_is_a_breakdown():
    b = _b()
    lab = synth.pool_scene(32, 1000)
    rhs = synth.rhs_normal(lab, 1001).astype(np.float32)
    for method in (1, 2):
        s = b.Solver(np.zeros(b.weight_count(4), np.float32), levels=4, method=method)
        _, _, _, st = s.solve(_dev(lab, torch.uint8), _dev(rhs, torch.float32), tol=1e-6, max_iter=10)
        assert st == b.BREAKDOWN
        s.close()


def test_bad_method_is_rejected():
    b = _b()
    with pytest.raises(b.NpsolveError):
        b.Solver(_trained(), levels=4, method=3)
