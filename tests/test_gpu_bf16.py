"""The BF16 form (the form bench.py times and the server runs) against the
oracle.

Two references:

* The oracle's model of the BF16 form (oracle.network(form="bf16"),
  PREC_NETWORK_BF16): the same folded weights and per-cell kernel values
  rounded to BF16, everything else in FP64.  The library evaluates exactly
  these rounded kernels with FP32 accumulation, so the tolerances are those
  of the FP32 form: the network output to 1e-5 norm-wise (and every entry to
  1e-5 of the largest), the NPSDO iteration count exactly where the oracle's
  stop is clear of the threshold (its last two residuals 5% or more either
  side of tol ||b||, else within one), and x to 1e-5 norm-wise.
* The exact FP64 oracle.  The rounding moves each kernel value by at most
  2^-8 relative, which moves the network output by 0.2-0.6% on these
  problems; it changes the preconditioner, not the system, so a converged
  BF16 solve and a converged FP64 solve both approximate the same x* = A^-1 b
  to the stop tolerance.  The stated bound: with eps the relative error of
  the oracle's own converged x against x* (x* from the oracle run to 1e-13),
  ||x_bf16 - x_oracle|| <= 3 eps ||x*|| (the BF16 x is no further from x* than
  twice the oracle's, plus the oracle's own error), and the BF16 count within
  3 of the FP64 one.
Measured (B300): network 0.9-2.2e-7 of the BF16 model; x 3e-8 - 8e-8 of the
BF16 model and 7.5e-8 - 7.1e-7 of the FP64 oracle, against eps = 1.8e-6 -
9.5e-6.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2310_00177_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2310_00177_b300", "weights", "npsdo_L4.f32")


def _b():
    from paper_2310_00177_b300 import binding

    return binding


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _rel(a, c):
    return float(np.linalg.norm(a - c) / max(np.linalg.norm(c), 1e-300))


def _rmc(lab, x):
    comp, pure = synth.neumann_components(lab)
    x = x.copy()
    for c in pure:
        m = comp == c
        x[m] -= x[m].mean()
    return x


def _rng_labels(shape, seed, p=(0.2, 0.6, 0.2)):
    return np.random.default_rng(seed).choice(np.array([0, 1, 2], np.uint8), size=shape, p=p)


NETS = [
    ("random 32^3, L=4", lambda: _rng_labels((32, 32, 32), 31), 4, lambda: synth.init_weights(4, 32, spread=0.05)),
    ("pool 32^3, L=4", lambda: synth.pool_scene(32, 1000), 4, lambda: synth.init_weights(4, 7)),
    ("ragged 24x40x56, L=4", lambda: _rng_labels((24, 40, 56), 5), 4, lambda: synth.init_weights(4, 32, spread=0.05)),
    ("ragged 16x32x48, L=3", lambda: _rng_labels((16, 32, 48), 6), 3, lambda: synth.init_weights(3, 8, spread=0.05)),
    ("slosh 64^3, L=5", lambda: synth.slosh_scene(64, 9), 5, lambda: synth.init_weights(5, 9)),
    ("slosh 64^3, trained L=4", lambda: synth.slosh_scene(64, 2000), 4, lambda: np.fromfile(WEIGHTS, np.float32)),
]


@pytest.mark.parametrize("case", range(len(NETS)), ids=[c[0] for c in NETS])
def test_bf16_network_matches_the_oracle_bf16_form(case):
    b = _b()
    _, mk_lab, L, mk_w = NETS[case]
    lab = mk_lab()
    w = np.asarray(mk_w(), np.float32)
    r = np.random.default_rng(33).standard_normal(lab.shape).astype(np.float32)
    zb = oracle.network(lab, L, w.astype(np.float64), r.astype(np.float64), form="bf16")
    zo = oracle.network(lab, L, w.astype(np.float64), r.astype(np.float64))
    e_form = _rel(zb, zo)
    assert 1e-4 < e_form < 2e-2  # the rounding is there and of its expected size
    for path in (b.PATH_CACHED, b.PATH_TENSOR, b.PATH_CUDA_CORE):
        s = b.Solver(w, levels=L, precision=b.BF16, kernel_path=path)
        z = s.apply_network(_dev(lab, torch.uint8), _dev(r, torch.float32)).cpu().numpy()
        s.close()
        assert _rel(z, zb) <= 1e-5, path
        assert np.abs(z - zb).max() <= 1e-5 * np.abs(zb).max(), path


SOLVES = [
    ("pool 32^3, seeded init", lambda: synth.pool_scene(32, 1000), 1001, lambda: synth.init_weights(4, 7), True),
    ("slosh 64^3, trained", lambda: synth.slosh_scene(64, 2000), 2001, lambda: np.fromfile(WEIGHTS, np.float32), True),
    ("slosh 64^3, seeded init (109 iterations)", lambda: synth.slosh_scene(64, 2000), 2001,
     lambda: synth.init_weights(4, 7), False),
]


def _count_ok(got, ores):
    h = ores["res_hist"] / ores["res_hist"][0]
    clear = h[-1] < 0.95e-6 and h[-2] > 1.05e-6
    return got == ores["iters"] if clear else abs(got - ores["iters"]) <= 1


@pytest.mark.parametrize("case", range(len(SOLVES)), ids=[c[0] for c in SOLVES])
def test_bf16_solve_matches_the_oracle(case):
    b = _b()
    _, mk_lab, seed, mk_w, against_exact = SOLVES[case]
    lab = mk_lab()
    rhs = synth.rhs_normal(lab, seed).astype(np.float32)
    w = np.asarray(mk_w(), np.float32)
    wd = w.astype(np.float64)
    obf = oracle.npsdo(lab, rhs.astype(np.float64), L=4, w=wd, tol=1e-6, max_iter=2000,
                       prec=oracle.PREC_NETWORK_BF16)
    s = b.Solver(w, levels=4, n_ortho=2, precision=b.BF16)
    x, iters, relres, st = s.solve(_dev(lab, torch.uint8), _dev(rhs, torch.float32), 1e-6, 2000)
    s.close()
    assert st == b.OK and relres < 1e-6
    assert _count_ok(iters, obf), (iters, obf["iters"])
    xg = _rmc(lab, x.cpu().numpy())
    assert _rel(xg, _rmc(lab, obf["x"])) <= 1e-5
    if against_exact:
        o64 = oracle.npsdo(lab, rhs.astype(np.float64), L=4, w=wd, tol=1e-6, max_iter=2000)
        ox = oracle.npsdo(lab, rhs.astype(np.float64), L=4, w=wd, tol=1e-13, max_iter=4000)
        xo, xs = _rmc(lab, o64["x"]), _rmc(lab, ox["x"])
        eps = _rel(xo, xs)
        assert 0 < eps < 1e-4
        assert _rel(xg, xs) <= 2 * eps
        assert np.linalg.norm(xg - xo) <= 3 * eps * np.linalg.norm(xs)
        assert abs(iters - o64["iters"]) <= 3
