"""Pins of the oracle's backward pass (reverse of Alg. 2) and of the training
loss gradient of Sec. 4.2.3.

CConv is bilinear in (kernel parameters, input vector), so the adjoint and the
parameter gradient satisfy exact identities; the full loss gradient is
checked against central finite differences in FP64 (step 1e-3)."""
import numpy as np
import pytest

import oracle
from paper_2310_00177_b300 import synth

S, F, A = 0, 1, 2


def _rng_labels(shape, seed, p=(0.3, 0.45, 0.25)):
    rng = np.random.default_rng(seed)
    return rng.choice(np.array([S, F, A], np.uint8), size=shape, p=p)


def test_cconv_adjoint_identity():
    rng = np.random.default_rng(0)
    lab = _rng_labels((5, 6, 7), 0)
    img = oracle.image(lab)
    W, B = rng.standard_normal((27, 3, 27)), rng.standard_normal(27)
    v, g = rng.standard_normal((2,) + lab.shape)
    gv, _, _ = oracle.cconv_backward(img, W, B, v, g)
    lhs = np.vdot(oracle.cconv(img, W, B, v), g)
    assert abs(lhs - np.vdot(v, gv)) < 1e-11 * abs(lhs)


def test_cconv_parameter_gradient_is_exact_for_bilinear_map():
    # <g, CConv_{W,B}(v)> is linear in (W, B): it equals <gW, W> + <gB, B>
    rng = np.random.default_rng(1)
    lab = _rng_labels((4, 5, 6), 1)
    img = oracle.image(lab)
    W, B = rng.standard_normal((27, 3, 27)), rng.standard_normal(27)
    v, g = rng.standard_normal((2,) + lab.shape)
    _, gW, gB = oracle.cconv_backward(img, W, B, v, g)
    lhs = np.vdot(oracle.cconv(img, W, B, v), g)
    assert abs(lhs - (np.vdot(gW, W) + np.vdot(gB, B))) < 1e-11 * abs(lhs)
    # and each block's gradient equals the output change per unit of that entry
    e = np.zeros((27, 3, 27))
    e[4, 1, 20] = 1.0
    assert np.vdot(oracle.cconv(img, e, np.zeros(27), v), g) == pytest.approx(gW[4, 1, 20], rel=1e-12)


def test_aff_gradient_is_exact():
    rng = np.random.default_rng(2)
    lab = _rng_labels((4, 4, 8), 2)
    img = oracle.image(lab)
    Wb = rng.standard_normal((3, 27))
    dW = oracle.aff_grad(img)
    assert oracle.aff(img, Wb, 0.4) == pytest.approx(0.4 + np.vdot(dW, Wb), rel=1e-13)


def test_network_input_gradient_is_the_adjoint():
    rng = np.random.default_rng(3)
    lab = _rng_labels((8, 8, 8), 3)
    w = rng.standard_normal(oracle.weight_count(4)) * 0.3
    r, gz = rng.standard_normal((2, 8, 8, 8))
    _, gr = oracle.network_backward(lab, 4, w, r, gz)
    lhs = np.vdot(oracle.network(lab, 4, w, r), gz)
    assert abs(lhs - np.vdot(r, gr)) < 1e-10 * abs(lhs)


@pytest.mark.parametrize("L", [1, 2, 4])
def test_network_weight_gradient_matches_finite_differences(L):
    rng = np.random.default_rng(4 + L)
    lab = _rng_labels((8, 8, 8), 4 + L)
    w = rng.standard_normal(oracle.weight_count(L)) * 0.2
    r, gz = rng.standard_normal((2, 8, 8, 8))
    gw, _ = oracle.network_backward(lab, L, w, r, gz)

    def f(wv):
        return np.vdot(oracle.network(lab, L, wv, r), gz)

    idx = rng.choice(w.size, size=24, replace=False)
    h = 1e-3
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (f(wp) - f(wm)) / (2 * h)
        assert fd == pytest.approx(gw[i], rel=1e-6, abs=1e-8 * np.abs(gw).max())


def test_loss_gradient_matches_finite_differences_16cubed():
    lab = synth.pool_scene(16, 21)
    b = synth.rhs_normal(lab, 22)
    b /= np.linalg.norm(b)
    w = synth.init_weights(4, 23, spread=0.05)
    loss, gw = oracle.loss(lab, 4, w, b)
    assert loss > 0
    rng = np.random.default_rng(24)
    # the largest-gradient entries plus random ones
    idx = np.concatenate([np.argsort(-np.abs(gw))[:6], rng.choice(w.size, 10, replace=False)])
    h = 1e-3

    def f(i, t):
        wt = w.copy()
        wt[i] += t
        return oracle.loss(lab, 4, wt, b, grad=False)

    for i in idx:
        # plain central difference (truncation error O(h^2)) ...
        fd2 = (f(i, h) - f(i, -h)) / (2 * h)
        assert fd2 == pytest.approx(gw[i], rel=1e-4, abs=1e-7 * np.abs(gw).max())
        # ... and the fourth-order central difference on the same step
        fd4 = (8 * (f(i, h) - f(i, -h)) - (f(i, 2 * h) - f(i, -2 * h))) / (12 * h)
        assert fd4 == pytest.approx(gw[i], rel=1e-7, abs=1e-9 * np.abs(gw).max())
