"""The network transpose, the asymmetry measure and the symmetric variant
P_sym,1 = P_net^T P_net (the paper's symmetry analysis, appendix): the CUDA
path through the C ABI against the FP64 oracle.

Tolerances: the transpose is a chain of FP32 CConv^T (27-term sums of
products with 55-term FP32 kernels), interpolation^T and pooling^T like the
forward network: norm-wise 1e-5.  S is a normalised difference of two FP32
dot products of size ~||x|| ||P y||, each correct to ~1e-7 relative: an
absolute error of 2e-5 plus 1e-3 S.  Solves: x after a fixed number of
iterations within 2e-5 (constants of pure-Neumann components removed); whole
solves converge and agree with the oracle's x through the residual (the
iteration count of the symmetric variant moves with FP32 rounding, see the
test)."""
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


@pytest.mark.parametrize("shape,L,path", [((32, 32, 32), 4, 0), ((24, 40, 56), 4, 1), ((6, 10, 14), 2, 0),
                                          ((16, 8, 24), 1, 0)])
def test_network_transpose_matches_oracle(shape, L, path):
    b = _b()
    lab = np.random.default_rng(61).choice(np.array([0, 1, 2], np.uint8), size=shape, p=(0.2, 0.6, 0.2))
    w = synth.init_weights(L, 62, spread=0.05).astype(np.float32)
    g = np.random.default_rng(63).standard_normal(shape).astype(np.float32)
    x = np.random.default_rng(64).standard_normal(shape).astype(np.float32)
    s = b.Solver(w, levels=L, kernel_path=path)
    lab_d = _dev(lab, torch.uint8)
    gt = s.network_transpose(lab_d, _dev(g, torch.float32)).cpu().numpy()
    go = oracle.network_transpose(lab, L, w.astype(np.float64), g.astype(np.float64))
    assert _rel(gt, go) <= 1e-5
    assert not gt[lab != 1].any()
    # adjoint identity against the library's own forward network
    px = s.apply_network(lab_d, _dev(x, torch.float32)).cpu().numpy().astype(np.float64)
    a, c = float((px * g).sum()), float((x.astype(np.float64) * gt).sum())
    assert abs(a - c) <= 1e-5 * (np.abs(px * g).sum())
    s.close()


@pytest.mark.parametrize("wkind", ["spread", "trained"])
def test_asymmetry_matches_oracle(wkind):
    b = _b()
    lab = synth.slosh_scene(32, 65)
    w = (synth.init_weights(4, 66, spread=0.05) if wkind == "spread" else _trained()).astype(np.float32)
    rng = np.random.default_rng(67)
    s = b.Solver(w, levels=4)
    lab_d = _dev(lab, torch.uint8)
    for _ in range(3):
        x = np.where(lab == 1, rng.standard_normal(lab.shape), 0.0).astype(np.float32)
        y = np.where(lab == 1, rng.standard_normal(lab.shape), 0.0).astype(np.float32)
        S, dots = s.asymmetry(lab_d, _dev(x, torch.float32), _dev(y, torch.float32))
        So = oracle.asymmetry(lab, 4, w.astype(np.float64), x.astype(np.float64), y.astype(np.float64))
        assert abs(S - So) <= 2e-5 + 1e-3 * So, (S, So)
    s.close()


@pytest.mark.parametrize("method", [0, 1, 2])
def test_symmetric_variant_solve_matches_oracle(method):
    b = _b()
    lab = synth.pool_scene(16, 26)
    rhs = synth.rhs_normal(lab, 27).astype(np.float32)
    w = _trained()
    kw = dict(L=4, w=w.astype(np.float64), tol=1e-6, max_iter=500, prec=oracle.PREC_NETWORK_SYM)
    if method == 0:
        ores = oracle.npsdo(lab, rhs.astype(np.float64), **kw)
    else:
        ores = oracle.npcg(lab, rhs.astype(np.float64), flexible=method == 2, **kw)
    assert ores["status"] == oracle.OK
    s = b.Solver(w, levels=4, method=method, symmetric=True)
    x, iters, relres, st = s.solve(_dev(lab, torch.uint8), _dev(rhs, torch.float32), tol=1e-6, max_iter=500)
    assert st == b.OK and relres < 1e-6
    # the count is not a stable observable here: P^T P squares the network's
    # conditioning, and in the oracle's own FP64 iteration a relative
    # perturbation of 1e-7 of the preconditioned vector (FP32 rounding) moves
    # it from 59 to 72 (NPSDO); so the bound is on the count, and x is compared
    # through the residual: both satisfy ||b - A x|| < tol ||b||
    assert ores["iters"] <= iters <= 1.35 * ores["iters"]
    xg = x.cpu().numpy()
    bm = np.where(lab == 1, rhs.astype(np.float64), 0.0)
    assert np.linalg.norm(oracle.lap_apply(lab, xg - ores["x"])) < 2e-6 * np.linalg.norm(bm)
    s.close()


@pytest.mark.parametrize("method", [0, 1])
def test_symmetric_variant_truncated_on_cached_path(method):
    # 32^3 at L = 4 runs the cached kernels; x after a fixed number of iterations
    b = _b()
    lab = synth.slosh_scene(32, 81)
    rhs = synth.rhs_normal(lab, 82).astype(np.float32)
    w = synth.init_weights(4, 83).astype(np.float32)
    s = b.Solver(w, levels=4, method=method, symmetric=True)
    for m in (1, 2, 3):
        kw = dict(L=4, w=w.astype(np.float64), tol=1e-12, max_iter=m, prec=oracle.PREC_NETWORK_SYM)
        ores = oracle.npsdo(lab, rhs.astype(np.float64), **kw) if method == 0 else \
            oracle.npcg(lab, rhs.astype(np.float64), **kw)
        x, iters, relres, st = s.solve(_dev(lab, torch.uint8), _dev(rhs, torch.float32), tol=1e-12, max_iter=m)
        assert st == b.NO_CONVERGENCE and iters == ores["iters"] == m
        assert _rel(_nc(lab, x.cpu().numpy()), _nc(lab, ores["x"])) <= 2e-5
    s.close()


def test_symmetric_variant_generic_path_truncated():
    b = _b()
    lab = np.random.default_rng(41).choice(np.array([0, 1, 2], np.uint8), size=(6, 10, 14), p=(0.15, 0.7, 0.15))
    rhs = synth.rhs_normal(lab, 42).astype(np.float32)
    w = synth.init_weights(2, 43).astype(np.float32)
    s = b.Solver(w, levels=2, method=b.PCG, symmetric=True)
    for m in (1, 4):
        ores = oracle.npcg(lab, rhs.astype(np.float64), L=2, w=w.astype(np.float64), tol=1e-12, max_iter=m,
                           prec=oracle.PREC_NETWORK_SYM)
        x, iters, relres, st = s.solve(_dev(lab, torch.uint8), _dev(rhs, torch.float32), tol=1e-12, max_iter=m)
        assert st == b.NO_CONVERGENCE and iters == m
        assert _rel(_nc(lab, x.cpu().numpy()), _nc(lab, ores["x"])) <= 2e-5
    s.close()
