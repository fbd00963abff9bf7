"""Pins of the oracle's PCG and flexible PCG with the network as
preconditioner (Sec. 4.1; the appendix's comparison of solver variants).

* A symmetric positive definite preconditioner reduces both to textbook PCG:
  the iterates equal scipy's ``cg`` with the same preconditioner, and the
  flexible (Polak-Ribiere) beta equals the Fletcher-Reeves one because
  z_k^T r_{k-1} = 0.
* With exact line search, flexible PCG's beta z_k^T (r_k - r_{k-1}) / rho_{k-1}
  equals -z_k^T A d_{k-1} / d_{k-1}^T A d_{k-1}, the A-orthogonalisation
  coefficient of Alg. 1 with one previous direction, for ANY preconditioner:
  flexible PCG with the (non-symmetric) network reproduces NPSDO with
  n_ortho = 1.
* The exact inverse converges in one step; a zero network breaks down."""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

import oracle
from paper_2310_00177_b300 import synth

F = 1


def _dense(lab):
    n = lab.size
    M = np.zeros((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        M[:, j] = oracle.lap_apply(lab, e.reshape(lab.shape)).ravel()
        e[j] = 0.0
    return M


def _scene(n, seed):
    lab = synth.pool_scene(n, seed)
    return lab, synth.rhs_normal(lab, seed + 1)


def _spd_preconditioner(lab, seed):
    # Jacobi plus a random symmetric positive semi-definite term, on fluid cells
    fl = (lab == F).ravel()
    M = _dense(lab)
    nf = int(fl.sum())
    g = np.random.default_rng(seed).standard_normal((nf, nf)) * (0.3 / nf)
    Pff = np.diag(1.0 / np.diag(M)[fl]) + g @ g.T
    P = np.zeros_like(M)
    P[np.ix_(fl, fl)] = Pff
    return M, P, fl


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("flexible", [False, True])
def test_spd_preconditioner_matches_scipy_cg(flexible):
    lab, b = _scene(8, 21)
    M, P, fl = _spd_preconditioner(lab, 22)
    Mff, Pff, bf = M[np.ix_(fl, fl)], P[np.ix_(fl, fl)], b.ravel()[fl]
    for m in (1, 2, 7):
        res = oracle.npcg(lab, b, prec=oracle.PREC_DENSE, pdense=P, tol=0.0, max_iter=m, flexible=flexible)
        assert res["status"] == oracle.NO_CONVERGENCE and res["iters"] == m
        xs, info = sla.cg(Mff, bf, x0=np.zeros_like(bf), rtol=0.0, atol=0.0, maxiter=m,
                          M=sla.LinearOperator(Mff.shape, matvec=lambda v: Pff @ v))
        x = res["x"].ravel()
        assert _rel(x[fl], xs) < 1e-10, m
        assert not x[~fl].any()


def test_identity_preconditioner_is_textbook_cg():
    lab, b = _scene(8, 23)
    M = _dense(lab)
    fl = (lab == F).ravel()
    Mff, bf = M[np.ix_(fl, fl)], b.ravel()[fl]
    res = oracle.npcg(lab, b, prec=oracle.PREC_IDENTITY, tol=0.0, max_iter=9)
    xs, _ = sla.cg(Mff, bf, x0=np.zeros_like(bf), rtol=0.0, atol=0.0, maxiter=9)
    assert _rel(res["x"].ravel()[fl], xs) < 1e-10


def test_flexible_equals_fletcher_reeves_for_symmetric_preconditioner():
    lab, b = _scene(8, 24)
    _, P, _ = _spd_preconditioner(lab, 25)
    r0 = oracle.npcg(lab, b, prec=oracle.PREC_DENSE, pdense=P, tol=1e-10, max_iter=200)
    r1 = oracle.npcg(lab, b, prec=oracle.PREC_DENSE, pdense=P, tol=1e-10, max_iter=200, flexible=True)
    assert r0["status"] == r1["status"] == oracle.OK and r0["iters"] == r1["iters"]
    np.testing.assert_allclose(r1["res_hist"], r0["res_hist"], rtol=1e-6)
    assert _rel(r1["x"], r0["x"]) < 1e-9


def test_network_is_not_symmetric():
    # the premise of the two tests below (Sec. 4.3 of the paper discusses the asymmetry)
    lab, _ = _scene(16, 26)
    w = synth.init_weights(4, 27, spread=0.05)
    rng = np.random.default_rng(28)
    u = np.where(lab == F, rng.standard_normal(lab.shape), 0.0)
    v = np.where(lab == F, rng.standard_normal(lab.shape), 0.0)
    a = float((u * oracle.network(lab, 4, w, v)).sum())
    c = float((v * oracle.network(lab, 4, w, u)).sum())
    assert abs(a - c) > 1e-3 * max(abs(a), abs(c))


def test_flexible_pcg_with_network_is_npsdo_with_one_orthogonalisation():
    lab, b = _scene(16, 26)
    w = synth.init_weights(4, 27, spread=0.05)
    for m in (1, 2, 5, 12):
        f = oracle.npcg(lab, b, L=4, w=w, tol=0.0, max_iter=m, flexible=True)
        s = oracle.npsdo(lab, b, L=4, w=w, tol=0.0, max_iter=m, n_ortho=1)
        assert f["iters"] == s["iters"] == m
        assert _rel(f["x"], s["x"]) < 1e-9, m
    # a whole solve, with the weights of the multilevel starting point
    w = synth.init_weights(4, 7)
    f = oracle.npcg(lab, b, L=4, w=w, tol=1e-8, max_iter=500, flexible=True)
    s = oracle.npsdo(lab, b, L=4, w=w, tol=1e-8, max_iter=500, n_ortho=1)
    assert f["status"] == s["status"] == oracle.OK and f["iters"] == s["iters"]
    assert f["relres"] < 1e-8
    np.testing.assert_allclose(f["res_hist"], s["res_hist"], rtol=1e-6)


def test_pcg_with_network_differs_from_flexible():
    # Fletcher-Reeves beta with a non-symmetric preconditioner: a different
    # method from the second direction on (the first step is the same)
    lab, b = _scene(16, 26)
    w = synth.init_weights(4, 27, spread=0.05)
    p1 = oracle.npcg(lab, b, L=4, w=w, tol=0.0, max_iter=1)
    f1 = oracle.npcg(lab, b, L=4, w=w, tol=0.0, max_iter=1, flexible=True)
    assert _rel(p1["x"], f1["x"]) < 1e-14
    p = oracle.npcg(lab, b, L=4, w=w, tol=0.0, max_iter=6)
    f = oracle.npcg(lab, b, L=4, w=w, tol=0.0, max_iter=6, flexible=True)
    assert _rel(p["x"], f["x"]) > 1e-6


def test_trained_network_variant_ordering():
    # the appendix's comparison of solver variants: with a trained network PCG
    # and flexible PCG both converge, and NPSDO (n_ortho = 2) needs no more
    # iterations than either (weights trained by paper_2310_00177_b300.train)
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    w = np.fromfile(os.path.join(here, "..", "paper_2310_00177_b300", "weights", "npsdo_L4.f32"), np.float32)
    lab, b = _scene(16, 26)
    p = oracle.npcg(lab, b, L=4, w=w, tol=1e-6, max_iter=300)
    f = oracle.npcg(lab, b, L=4, w=w, tol=1e-6, max_iter=300, flexible=True)
    s = oracle.npsdo(lab, b, L=4, w=w, tol=1e-6, max_iter=300)
    assert p["status"] == f["status"] == s["status"] == oracle.OK
    assert s["iters"] <= f["iters"] <= p["iters"]


def test_exact_inverse_converges_in_one_step():
    lab, b = _scene(8, 29)
    fl = (lab == F).ravel()
    M = _dense(lab)
    P = np.zeros_like(M)
    P[np.ix_(fl, fl)] = np.linalg.inv(M[np.ix_(fl, fl)])
    for flexible in (False, True):
        res = oracle.npcg(lab, b, prec=oracle.PREC_DENSE, pdense=P, tol=1e-10, max_iter=10, flexible=flexible)
        assert res["iters"] == 1 and res["relres"] < 1e-12


def test_zero_network_breaks_down():
    lab, b = _scene(8, 30)
    for flexible in (False, True):
        res = oracle.npcg(lab, b, L=2, w=np.zeros(oracle.weight_count(2)), max_iter=5, flexible=flexible)
        assert res["status"] == oracle.BREAKDOWN and res["iters"] == 1


@pytest.mark.parametrize("flexible", [False, True])
def test_explicit_and_recurrence_residual_modes_agree(flexible):
    # R2 for the PCG variants: r_k = b - A x_k or the recurrence give the same
    # iterates up to rounding; both converge and their counts differ by at most one
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    w = np.fromfile(os.path.join(here, "..", "paper_2310_00177_b300", "weights", "npsdo_L4.f32"), np.float32)
    lab, b = _scene(16, 26)
    r0 = oracle.npcg(lab, b, L=4, w=w, tol=1e-6, max_iter=300, flexible=flexible, residual_mode=0)
    r1 = oracle.npcg(lab, b, L=4, w=w, tol=1e-6, max_iter=300, flexible=flexible, residual_mode=1)
    assert r0["status"] == r1["status"] == oracle.OK and abs(r0["iters"] - r1["iters"]) <= 1
    assert r0["relres"] < 1e-6 and r1["relres"] < 1e-6
    m = min(r0["iters"], r1["iters"])
    np.testing.assert_allclose(r0["res_hist"][:m], r1["res_hist"][:m], rtol=1e-6)
