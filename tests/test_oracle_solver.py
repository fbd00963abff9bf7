"""Pins of the oracle's NPSDO (Sec. 4.1, Alg. 1) and Jacobi-PCG.

Sec. 4.1 states the reductions used here: with the identity preconditioner
and n_ortho >= 1 the method is unpreconditioned CG, with n_ortho = 0 it is
steepest descent, and with the exact inverse it converges in one step.  The
converged solution is also compared with a dense direct solve."""
import numpy as np
import pytest

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


def _scene(n=8, seed=3):
    lab = synth.pool_scene(n, seed)
    b = synth.rhs_normal(lab, seed + 1)
    return lab, b


def textbook_cg(M, b, tol, max_iter):
    """Hestenes-Stiefel CG on a dense SPD(-on-range) matrix."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = r @ r
    nb = np.sqrt(rr)
    hist = [nb]
    k = 0
    while np.sqrt(rr) >= tol * nb and k < max_iter:
        k += 1
        q = M @ p
        a = rr / (p @ q)
        x += a * p
        r -= a * q
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
        hist.append(np.sqrt(rr))
    return x, k, np.array(hist)


def textbook_sd(M, b, iters):
    x = np.zeros_like(b)
    r = b.copy()
    for _ in range(iters):
        q = M @ r
        x += (r @ r) / (r @ q) * r
        r = b - M @ x
    return x


@pytest.mark.parametrize("n_ortho", [1, 2, 3])
def test_identity_preconditioner_is_cg(n_ortho):
    lab, b = _scene(8, 3)
    M = _dense(lab)
    xcg, kcg, hcg = textbook_cg(M, b.ravel(), 1e-6, 500)
    res = oracle.npsdo(lab, b, prec=oracle.PREC_IDENTITY, tol=1e-6, max_iter=500, n_ortho=n_ortho)
    assert res["iters"] == kcg
    np.testing.assert_allclose(res["res_hist"], hcg, rtol=1e-6, atol=1e-12 * hcg[0])
    np.testing.assert_allclose(res["x"].ravel(), xcg, rtol=1e-8, atol=1e-9 * np.abs(xcg).max())


def test_identity_preconditioner_without_orthogonalization_is_steepest_descent():
    lab, b = _scene(8, 4)
    M = _dense(lab)
    res = oracle.npsdo(lab, b, prec=oracle.PREC_IDENTITY, tol=0.0, max_iter=15, n_ortho=0)
    assert res["status"] == oracle.NO_CONVERGENCE and res["iters"] == 15
    xsd = textbook_sd(M, b.ravel(), 15)
    np.testing.assert_allclose(res["x"].ravel(), xsd, rtol=1e-9, atol=1e-11 * np.abs(xsd).max())


def test_exact_inverse_converges_in_one_step():
    lab, b = _scene(8, 5)
    fl = (lab == F).ravel()
    M = _dense(lab)
    P = np.zeros_like(M)
    P[np.ix_(fl, fl)] = np.linalg.inv(M[np.ix_(fl, fl)])
    res = oracle.npsdo(lab, b, prec=oracle.PREC_DENSE, pdense=P, tol=1e-10, max_iter=10)
    assert res["iters"] == 1 and res["relres"] < 1e-12


def test_network_solve_converges_to_dense_solution():
    lab, b = _scene(16, 6)
    _, pure = synth.neumann_components(lab)
    assert len(pure) == 0
    fl = (lab == F).ravel()
    M = _dense(lab)[np.ix_(fl, fl)]
    xd = np.linalg.solve(M, b.ravel()[fl])
    w = synth.init_weights(4, 7)
    res = oracle.npsdo(lab, b, L=4, w=w, tol=1e-12, max_iter=500)
    assert res["status"] == oracle.OK and res["relres"] < 1e-12
    x = res["x"].ravel()
    np.testing.assert_allclose(x[fl], xd, rtol=0, atol=1e-9 * np.abs(xd).max())
    assert not x[~fl].any()


def test_energy_error_decreases_monotonically():
    # exact line search along each d_k: the A-norm of the error never grows
    lab, b = _scene(16, 7)
    fl = (lab == F).ravel()
    M = _dense(lab)[np.ix_(fl, fl)]
    xd = np.linalg.solve(M, b.ravel()[fl])
    w = synth.init_weights(4, 8, spread=0.05)
    errs = []
    for k in range(0, 12):
        x = oracle.npsdo(lab, b, L=4, w=w, tol=0.0, max_iter=k)["x"].ravel()[fl]
        e = x - xd
        errs.append(e @ M @ e)
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))


def test_residual_decreases_far_below_tolerance_in_fp64():
    # Sec. 5 appendix "Capacity for residual reduction": with the solver in
    # double precision, 100 iterations without a convergence test drive the
    # relative residual to about 1e-15.
    lab, b = _scene(16, 9)
    w = synth.init_weights(4, 9)
    res = oracle.npsdo(lab, b, L=4, w=w, tol=0.0, max_iter=100)
    assert res["relres"] < 1e-12


def test_explicit_and_recurrence_residual_modes_agree():
    lab = synth.pool_scene(32, 1000)
    b = synth.rhs_normal(lab, 1001)
    w = synth.init_weights(4, 7)
    r0 = oracle.npsdo(lab, b, L=4, w=w, residual_mode=0)
    r1 = oracle.npsdo(lab, b, L=4, w=w, residual_mode=1)
    assert abs(r0["iters"] - r1["iters"]) <= 1
    assert r0["relres"] < 1e-6 and r1["relres"] < 1e-6


def test_pure_neumann_components_converge_modulo_constants():
    # two fluid pockets sealed by solid (pure Neumann) plus an open region
    lab = synth.pool_scene(16, 11)
    lab[2:6, 2:6, 2:6] = 0
    lab[3:5, 3:5, 3:5] = F
    b = synth.rhs_normal(lab, 12)
    comp, pure = synth.neumann_components(lab)
    assert len(pure) >= 1
    res = oracle.npsdo(lab, b, L=4, w=synth.init_weights(4, 7), tol=1e-10, max_iter=800)
    assert res["status"] == oracle.OK and res["relres"] < 1e-10


def test_jacobi_pcg_matches_textbook_pcg():
    lab, b = _scene(8, 13)
    M = _dense(lab)
    dg = np.diag(M).copy()
    inv = np.where(dg > 0, 1.0 / np.where(dg > 0, dg, 1), 0.0)
    x = np.zeros(lab.size)
    r = b.ravel().copy()
    z = inv * r
    p = z.copy()
    rz = r @ z
    k = 0
    nb = np.linalg.norm(r)
    while np.linalg.norm(r) >= 1e-8 * nb:
        k += 1
        q = M @ p
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        z = inv * r
        rz2 = r @ z
        p = z + rz2 / rz * p
        rz = rz2
    res = oracle.jacobi_pcg(lab, b, tol=1e-8)
    assert res["iters"] == k
    np.testing.assert_allclose(res["x"].ravel(), x, rtol=1e-9, atol=1e-10 * np.abs(x).max())


def test_zero_network_breaks_down_and_nan_rhs_is_rejected():
    lab, b = _scene(8, 14)
    res = oracle.npsdo(lab, b, L=2, w=np.zeros(oracle.weight_count(2)), max_iter=5)
    assert res["status"] == oracle.BREAKDOWN
    bad = b.copy()
    bad[tuple(np.argwhere(lab == F)[0])] = np.nan
    with pytest.raises(ValueError):
        oracle.npsdo(lab, bad, L=2, w=synth.init_weights(2, 1))
