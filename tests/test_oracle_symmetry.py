"""Pins of the oracle's symmetry tools (the appendix's analysis and
enforcement of symmetry): the asymmetry measure
S(x, y; I) = |x.P(y) - y.P(x)| / sqrt(|x.P(x)| |y.P(y)|), the network
transpose and the symmetric variant P_sym,1 = P_net^T P_net as a
preconditioner."""
import numpy as np
import scipy.sparse.linalg as sla

import oracle
from paper_2310_00177_b300 import synth

F = 1


def _vecs(lab, seed):
    rng = np.random.default_rng(seed)
    return [np.where(lab == F, rng.standard_normal(lab.shape), 0.0) for _ in range(2)]


def _conv_weights(B):
    # L = 1 with W = 0: the network is the masked, zero-padded convolution with the 27 taps B
    w = np.zeros(oracle.weight_count(1))
    w[27 * 3 * 27:] = B
    return w


def test_asymmetry_measure_basic_properties():
    lab = synth.pool_scene(16, 31)
    w = synth.init_weights(4, 32, spread=0.05)
    x, y = _vecs(lab, 33)
    s = oracle.asymmetry(lab, 4, w, x, y)
    assert s > 1e-4
    assert abs(oracle.asymmetry(lab, 4, w, y, x) - s) < 1e-12 * s
    assert abs(oracle.asymmetry(lab, 4, w, 2.0 * x, -3.0 * y) - s) < 1e-10 * s
    assert oracle.asymmetry(lab, 4, w, x, x) < 1e-14


def test_symmetric_taps_give_zero_asymmetry():
    # B_a = B_{-a}: the convolution equals its transpose (tap t and 26 - t are opposite offsets)
    lab = synth.pool_scene(16, 34)
    B = np.random.default_rng(35).standard_normal(27)
    B = 0.5 * (B + B[::-1])
    x, y = _vecs(lab, 36)
    assert oracle.asymmetry(lab, 1, _conv_weights(B), x, y) < 1e-13


def test_single_tap_asymmetry_closed_form():
    # B = e_t: P v(p) = v(p + a) on fluid, zero-padded; x.P(y) = sum_p x(p) y(p + a)
    lab = synth.pool_scene(16, 37)
    t = 9 * 2 + 3 * 1 + 0  # offset (dz, dy, dx) = (+1, 0, -1)
    B = np.zeros(27)
    B[t] = 1.0
    x, y = _vecs(lab, 38)

    def shift(v):  # v(p + a) with a = (+1, 0, -1), zero outside
        o = np.zeros_like(v)
        o[:-1, :, 1:] = v[1:, :, :-1]
        return o

    fl = lab == F
    px, py = np.where(fl, shift(x), 0.0), np.where(fl, shift(y), 0.0)
    want = abs((x * py).sum() - (y * px).sum()) / np.sqrt(abs((x * px).sum()) * abs((y * py).sum()))
    got = oracle.asymmetry(lab, 1, _conv_weights(B), x, y)
    assert abs(got - want) < 1e-12 * want


def test_network_transpose_is_the_adjoint():
    lab = synth.slosh_scene(16, 39)
    w = synth.init_weights(4, 40, spread=0.05)
    x, y = _vecs(lab, 41)
    a = float((oracle.network(lab, 4, w, x) * y).sum())
    b = float((x * oracle.network_transpose(lab, 4, w, y)).sum())
    assert abs(a - b) < 1e-12 * abs(a)


def test_symmetric_variant_is_symmetric_positive_semidefinite():
    lab = synth.slosh_scene(16, 42)
    w = synth.init_weights(4, 43, spread=0.05)
    x, y = _vecs(lab, 44)

    def psym(v):
        return oracle.network_transpose(lab, 4, w, oracle.network(lab, 4, w, v))

    xpy, ypx = float((x * psym(y)).sum()), float((y * psym(x)).sum())
    assert abs(xpy - ypx) < 1e-12 * abs(xpy)
    assert float((x * psym(x)).sum()) > 0 and float((y * psym(y)).sum()) > 0


def test_pcg_with_symmetric_variant_matches_scipy_cg():
    # P_sym is symmetric positive (semi)definite: PCG with it is textbook PCG,
    # compared with scipy's cg on the dense fluid block after a few steps
    lab = synth.pool_scene(8, 45)
    b = synth.rhs_normal(lab, 46)
    w = synth.init_weights(2, 47)
    fl = (lab == F).ravel()
    n = lab.size
    Pd = np.zeros((n, n))
    M = np.zeros((n, n))
    e = np.zeros(n)
    for j in np.flatnonzero(fl):
        e[j] = 1.0
        v = e.reshape(lab.shape)
        Pd[:, j] = oracle.network_transpose(lab, 2, w, oracle.network(lab, 2, w, v)).ravel()
        M[:, j] = oracle.lap_apply(lab, v).ravel()
        e[j] = 0.0
    Mff, Pff, bf = M[np.ix_(fl, fl)], Pd[np.ix_(fl, fl)], b.ravel()[fl]
    for m in (1, 3, 6):
        res = oracle.npcg(lab, b, L=2, w=w, prec=oracle.PREC_NETWORK_SYM, tol=0.0, max_iter=m)
        xs, _ = sla.cg(Mff, bf, x0=np.zeros_like(bf), rtol=0.0, atol=0.0, maxiter=m,
                       M=sla.LinearOperator(Mff.shape, matvec=lambda v: Pff @ v))
        x = res["x"].ravel()
        assert np.linalg.norm(x[fl] - xs) < 1e-9 * np.linalg.norm(xs), m


def test_symmetric_variant_of_trained_network_needs_more_iterations():
    # the appendix reports the symmetric variants preconditioning worse than the
    # proposed network; built from the trained P_net (approximating A^-1),
    # P^T P approximates A^-2
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    w = np.fromfile(os.path.join(here, "..", "paper_2310_00177_b300", "weights", "npsdo_L4.f32"), np.float32)
    lab = synth.pool_scene(16, 26)
    b = synth.rhs_normal(lab, 27)
    p = oracle.npsdo(lab, b, L=4, w=w, tol=1e-6, max_iter=300)
    s = oracle.npcg(lab, b, L=4, w=w, tol=1e-6, max_iter=300, prec=oracle.PREC_NETWORK_SYM)
    assert p["status"] == s["status"] == oracle.OK and s["iters"] > 2 * p["iters"]
