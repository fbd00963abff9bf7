"""The hand-written backward (reverse of Alg. 2) and the training loss of
Sec. 4.2.3 on the GPU against the FP64 oracle and finite differences.

Tolerances: the GPU backward accumulates the weight gradient in FP32 (on the
tensor cores for levels 1-3: the kernel gradient as three BF16 terms, exact
features, FP32 accumulation per CTA; FP32 CUDA-core batches beyond) and in
FP64 across CTAs; for a 16^3 grid each weight-gradient entry is a sum of
O(10^4) products, so its rounding error is ~sqrt(10^4) eps32 ~ 1e-5 of the sum
of magnitudes.  Norm-wise relative error <= 1e-4 and element-wise
<= 1e-4 * max|g| against the FP64 oracle gradient.  The finite-difference
check (central, step 1e-3, FP64, oracle loss) is limited by the O(h^2)
truncation: relative 1e-3 on the largest entries."""
import numpy as np
import pytest

import oracle
from paper_2310_00177_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _b():
    from paper_2310_00177_b300 import binding

    return binding


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _rng_labels(shape, seed, p=(0.2, 0.6, 0.2)):
    rng = np.random.default_rng(seed)
    return rng.choice(np.array([0, 1, 2], np.uint8), size=shape, p=p)


# (nz, ny, nx): rows of a multiple of 8 cells take the 8-cell-run operand
# staging of the tensor-core weight gradient, others the per-cell one; 10 x 22
# x 24 and 16 x 24 x 40 span tens of 128-cell chunks, the first with a partial
# last one.  Rows of a multiple of 32 cells take the forward on the tensor
# cores at levels 1-3 (4 x 8 x 64: levels 1 and 2; 8 x 8 x 256: levels 1-3)
# and the CUDA-core forward with row loads beyond (8 x 8 x 256: level 4, 32
# cells wide); the rest the CUDA-core forward with per-cell loads.
@pytest.mark.parametrize("shape,L", [((16, 16, 16), 4), ((8, 16, 24), 3), ((8, 8, 8), 1), ((16, 8, 16), 2),
                                     ((10, 22, 24), 2), ((16, 24, 40), 3), ((4, 8, 64), 2), ((8, 8, 256), 4)])
def test_network_vjp_matches_oracle_backward(shape, L):
    b = _b()
    lab = _rng_labels(shape, 61) if shape != (16, 16, 16) else synth.pool_scene(16, 62)
    w = synth.init_weights(L, 63, spread=0.05).astype(np.float32)
    rng = np.random.default_rng(64)
    r = rng.standard_normal(shape).astype(np.float32)
    gz = rng.standard_normal(shape).astype(np.float32)
    s = b.Solver(w, levels=L)
    gw, gr = s.network_vjp(_dev(lab, torch.uint8), _dev(r, torch.float32), _dev(gz, torch.float32))
    ogw, ogr = oracle.network_backward(lab, L, w.astype(np.float64), r.astype(np.float64), gz.astype(np.float64))
    assert _rel(gw, ogw) <= 1e-4
    assert np.abs(gw - ogw).max() <= 1e-4 * np.abs(ogw).max()
    assert _rel(gr.cpu().numpy(), ogr) <= 1e-5
    s.close()


def test_misaligned_device_pointers_are_rejected():
    """The kernels use 8- and 16-byte vector accesses: an offset view is
    refused at the boundary, before anything is launched on it."""
    b = _b()
    shape = (8, 8, 8)
    lab = synth.pool_scene(8, 62)
    n = lab.size
    big = torch.zeros(n + 16, dtype=torch.uint8, device="cuda")
    big[1:n + 1] = _dev(lab.ravel(), torch.uint8)
    lab_off = big[1:n + 1].view(shape)
    assert lab_off.data_ptr() % 16 == 1 and lab_off.is_contiguous()
    rng = np.random.default_rng(5)
    r = _dev(rng.standard_normal(shape), torch.float32)
    s = b.Solver(synth.init_weights(2, 7).astype(np.float32), levels=2)
    with pytest.raises(b.NpsolveError, match="16-byte aligned"):
        s.solve(lab_off, r, 1e-6, 10)
    with pytest.raises(b.NpsolveError, match="16-byte aligned"):
        s.network_vjp(lab_off, r, r)
    with pytest.raises(b.NpsolveError, match="16-byte aligned"):
        s.train_step([lab_off], [r], lr=1e-3)
    # the handle still works with aligned arguments
    _, it, rr, st = s.solve(_dev(lab, torch.uint8), r, 1e-6, 200)
    assert st == b.OK and rr < 1e-6
    s.close()


def test_network_vjp_adjoint_identity():
    # P_net is linear in r: <gz, P(r)> = <gr, r>
    b = _b()
    lab = synth.slosh_scene(32, 71)
    w = synth.init_weights(4, 72, spread=0.05).astype(np.float32)
    rng = np.random.default_rng(73)
    r = _dev(rng.standard_normal(lab.shape), torch.float32)
    gz = _dev(rng.standard_normal(lab.shape), torch.float32)
    labd = _dev(lab, torch.uint8)
    s = b.Solver(w)
    z = s.apply_network(labd, r)
    _, gr = s.network_vjp(labd, r, gz)
    mask = labd == 1
    lhs = float((gz.double() * z.double()).sum())
    rhs = float((gr.double() * torch.where(mask, r, 0).double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    s.close()


def test_loss_gradient_matches_oracle_and_finite_differences_16cubed():
    # the configuration's check: central differences, step 1e-3, FP64, 16^3
    b = _b()
    lab = synth.pool_scene(16, 21)
    rhs = synth.rhs_normal(lab, 22)
    rhs = (rhs / np.linalg.norm(rhs)).astype(np.float32)
    w = synth.init_weights(4, 23, spread=0.05).astype(np.float32)
    s = b.Solver(w)
    loss, gw = s.loss_grad(_dev(lab, torch.uint8), _dev(rhs, torch.float32))
    oloss, ogw = oracle.loss(lab, 4, w.astype(np.float64), rhs.astype(np.float64))
    assert loss == pytest.approx(oloss, rel=1e-5)
    assert _rel(gw, ogw) <= 1e-4
    idx = np.argsort(-np.abs(ogw))[:8]
    h = 1e-3
    for i in idx:
        wp, wm = w.astype(np.float64), w.astype(np.float64)
        wp = wp.copy()
        wm = wm.copy()
        wp[i] += h
        wm[i] -= h
        fd = (oracle.loss(lab, 4, wp, rhs.astype(np.float64), grad=False)
              - oracle.loss(lab, 4, wm, rhs.astype(np.float64), grad=False)) / (2 * h)
        assert gw[i] == pytest.approx(fd, rel=1e-3, abs=1e-6 * np.abs(ogw).max())
    s.close()


def test_autograd_function_uses_the_handwritten_backward():
    b = _b()
    lab = synth.pool_scene(16, 31)
    w = synth.init_weights(4, 32, spread=0.05).astype(np.float32)
    rng = np.random.default_rng(33)
    r = _dev(rng.standard_normal(lab.shape), torch.float32).requires_grad_(True)
    wt = torch.from_numpy(w).requires_grad_(True)
    labd = _dev(lab, torch.uint8)
    s = b.Solver(w)
    z = b.NetworkFunction.apply(wt, labd, r, s)
    gz = _dev(rng.standard_normal(lab.shape), torch.float32)
    (z * gz).sum().backward()
    ogw, ogr = oracle.network_backward(lab, 4, w.astype(np.float64), r.detach().cpu().numpy().astype(np.float64),
                                       gz.cpu().numpy().astype(np.float64))
    assert _rel(wt.grad.numpy(), ogw) <= 1e-4
    assert _rel(r.grad.cpu().numpy(), ogr) <= 1e-5
    s.close()


def test_train_step_reduces_the_loss():
    b = _b()
    labs, bs = [], []
    for i in range(4):
        lab = synth.slosh_scene(32, 400 + i)
        rhs = synth.rhs_normal(lab, 500 + i)
        labs.append(_dev(lab, torch.uint8))
        bs.append(_dev(rhs / np.linalg.norm(rhs), torch.float32))
    s = b.Solver(synth.init_weights(4, 7).astype(np.float32))
    losses = [s.train_step(labs, bs, lr=1e-3) for _ in range(30)]
    assert losses[-1] < 0.9 * losses[0]
    assert all(np.isfinite(losses))
    s.close()


def test_lanczos_ritz_values_match_dense_eigenvalues():
    # on a small grid the lowest Ritz values of a long Lanczos run converge
    # to the lowest eigenvalues of the reduced matrix (dense FP64 eigvalsh)
    b = _b()
    lab = synth.pool_scene(8, 3)
    fl = (lab == 1).ravel()
    n = lab.size
    M = np.zeros((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        M[:, j] = oracle.lap_apply(lab, e.reshape(lab.shape)).ravel()
        e[j] = 0.0
    ev = np.linalg.eigvalsh(M[np.ix_(fl, fl)])
    start = synth.rhs_normal(lab, 4).astype(np.float32)
    rhs, vals = b.lanczos_rhs(_dev(lab, torch.uint8), _dev(start, torch.float32), m=min(120, int(fl.sum())), k=4,
                              count=3, seed=5)
    np.testing.assert_allclose(vals, ev[:4], rtol=1e-4)
    r = rhs.cpu().numpy()
    assert np.allclose(np.linalg.norm(r.reshape(3, -1), axis=1), 1.0, atol=1e-4)
    assert not r[:, lab != 1].any()


def test_lanczos_at_the_papers_scale():
    # 1600 Lanczos steps with full reorthogonalisation and 800 combinations of
    # all 1600 Ritz vectors (the paper's training recipe, Sec. 4.2.3) on a
    # 2051-unknown system: the extreme Ritz values have converged to the
    # extreme eigenvalues of the reduced matrix (dense FP64 eigvalsh), every
    # Ritz value lies inside the spectrum, and the combinations are unit
    # vectors on the fluid cells.
    b = _b()
    lab = synth.pool_scene(16, 3)
    fl = (lab == 1).ravel()
    n = lab.size
    M = np.zeros((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        M[:, j] = oracle.lap_apply(lab, e.reshape(lab.shape)).ravel()
        e[j] = 0.0
    ev = np.linalg.eigvalsh(M[np.ix_(fl, fl)])
    start = synth.rhs_normal(lab, 4).astype(np.float32)
    m = 1600
    rhs, vals = b.lanczos_rhs(_dev(lab, torch.uint8), _dev(start, torch.float32), m=m, k=m, count=800, seed=5)
    assert vals.shape == (m,) and np.all(np.diff(vals) >= 0)
    np.testing.assert_allclose(vals[:8], ev[:8], rtol=1e-4)
    np.testing.assert_allclose(vals[-8:], ev[-8:], rtol=1e-4)
    assert ev[0] * (1 - 1e-4) <= vals[0] and vals[-1] <= ev[-1] * (1 + 1e-4)
    r = rhs.cpu().numpy().reshape(800, -1)
    np.testing.assert_allclose(np.linalg.norm(r, axis=1), 1.0, atol=2e-4)
    assert not r[:, ~fl].any()
