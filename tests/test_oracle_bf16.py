"""Pins of the oracle's BF16 form (the CUDA library's NPSOLVE_BF16 setting).

The form is the network of Alg. 2 with every CConv kernel value rounded to
BF16, after the exact rewrite of the kernel by the channel-sum identity
I_solid = 1 - I_fluid - I_air (Sec. 3.2) into folded weights over integer
fluid / air counts, whose folded weights are rounded to BF16 too.  Pins:

* the rounding itself against torch's FP32 -> BF16 conversion (a library
  routine), ties and the FP64 -> FP32 step included;
* weights whose folded values and per-cell kernels are all exactly
  representable in BF16: the BF16 form must equal the exact CConv, so any
  mistake in the fold (a dropped solid term, a wrong sign or channel, a wrong
  1/8^(l-1) scale) shows;
* general weights: every BF16-form kernel value is a BF16 number, and differs
  from the exact kernel by no more than the rounding bound (2^-8 relative per
  rounded weight and per kernel value);
* a second derivation of the BF16-form kernels with NumPy and torch's
  rounding;
* the BF16-form network is still linear in r, reduces to one BF16 CConv at
  L = 1, and the BF16-form NPSDO solve reaches the tolerance.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_00177_b300 import synth

S, F, A = 0, 1, 2
EPS_BF16 = 2.0 ** -8  # unit roundoff of an 8-significant-bit format (half its 2^-7 spacing at 1)


def _torch_bf16(v):
    t = torch.from_numpy(np.asarray(v, np.float64)).to(torch.float32).to(torch.bfloat16)
    return t.to(torch.float64).numpy()


def _rng_labels(shape, seed, p=(0.3, 0.45, 0.25)):
    rng = np.random.default_rng(seed)
    return rng.choice(np.array([S, F, A], np.uint8), size=shape, p=p)


def test_round_bf16_matches_torch_conversion():
    rng = np.random.default_rng(0)
    v = np.concatenate([
        rng.standard_normal(3000) * 10.0 ** rng.integers(-30, 30, 3000),
        rng.uniform(-1, 1, 2000),
    ])
    # exact ties between two BF16 neighbours, both parities of the kept bit
    base = _torch_bf16(rng.uniform(1, 2, 500))
    ties = base + np.ldexp(1.0, -8)  # half a BF16 step at [1, 2)
    # values within FP64 of a tie: the FP32 step decides
    near = ties + np.ldexp(1.0, -40) * rng.choice([-1.0, 1.0], 500)
    v = np.concatenate([v, ties, -ties, near, [0.0, -0.0, 1.0, 3.0e38, 1e-40, -1e-39]])
    np.testing.assert_array_equal(oracle.round_bf16(v), _torch_bf16(v))


def _exact_weights(rng, lvl):
    """Sparse weights on a dyadic grid, so that the folded weights and every
    kernel are exactly representable with 8 significant bits.  The image of
    level lvl holds multiples of 1/F, F = 8^(lvl-1).  Level 1: two entries
    of +-1 or +-2 steps of 2^-4 per tap and a bias of up to 4 steps, so every
    kernel is a multiple of 2^-4 below 2^4.  Coarser levels: one such entry
    per tap and no bias, so a kernel is (entry) x count / F, at most 2F
    multiples of 2^-4 / F."""
    W = np.zeros((27, 3, 27))
    step = 2.0 ** -4
    for a in range(27):
        for _ in range(2 if lvl == 1 else 1):
            W[a, rng.integers(0, 3), rng.integers(0, 27)] = step * rng.choice([-2, -1, 1, 2])
    B = step * rng.integers(-4, 5, 27) if lvl == 1 else np.zeros(27)
    return W, B


@pytest.mark.parametrize("lvl", [1, 2, 3])
def test_bf16_form_equals_exact_cconv_for_representable_weights(lvl):
    rng = np.random.default_rng(10 + lvl)
    lab = _rng_labels((8 << (lvl - 1),) * 3, 20 + lvl)
    img = oracle.image(lab)
    for _ in range(lvl - 1):
        img = oracle.avgpool2(img)
    W, B = _exact_weights(rng, lvl)
    K = oracle.cconv_kernels(img, W, B)
    assert np.array_equal(oracle.round_bf16(K), K)  # the construction keeps the kernels exact
    Kb = oracle.cconv_kernels_bf16(img, W, B, lvl)
    np.testing.assert_array_equal(Kb, K)
    v = rng.standard_normal(img.shape[1:])
    np.testing.assert_allclose(oracle.cconv_bf16(img, W, B, v, lvl), oracle.cconv(img, W, B, v), rtol=0, atol=1e-13)


@pytest.mark.parametrize("lvl", [1, 2, 4])
def test_bf16_form_kernels_are_bf16_within_the_rounding_bound(lvl):
    rng = np.random.default_rng(30 + lvl)
    lab = _rng_labels((8 << (lvl - 1),) * 3, 40 + lvl)
    img = oracle.image(lab)
    for _ in range(lvl - 1):
        img = oracle.avgpool2(img)
    W = rng.uniform(-0.2, 0.2, (27, 3, 27))
    B = rng.uniform(-0.5, 0.5, 27)
    K = oracle.cconv_kernels(img, W, B)
    Kb = oracle.cconv_kernels_bf16(img, W, B, lvl)
    assert np.array_equal(oracle.round_bf16(Kb), Kb)
    assert (Kb != K).mean() > 0.5  # the rounding is not vacuous
    # bound: each folded weight and the folded bias carry a relative error of
    # at most u = 2^-8 (plus FP32's 2^-24 before it), the kernel value another u
    Fc = 8.0 ** (lvl - 1)
    Wf = (W[:, 0, :] - W[:, 2, :]) / Fc
    Wa = (W[:, 1, :] - W[:, 2, :]) / Fc
    Bp = B + W[:, 2, :].sum(axis=1)
    nF = np.zeros(img.shape[1:] + (27,))
    nA = np.zeros_like(nF)
    pf = np.pad(img[0], 1)  # padding: solid, no fluid or air
    pa = np.pad(img[1], 1)
    nz, ny, nx = img.shape[1:]
    for t in range(27):
        dz, dy, dx = t // 9, (t // 3) % 3, t % 3
        nF[..., t] = Fc * pf[dz:dz + nz, dy:dy + ny, dx:dx + nx]
        nA[..., t] = Fc * pa[dz:dz + nz, dy:dy + ny, dx:dx + nx]
    Ssum = np.abs(Bp) + np.abs(nF) @ np.abs(Wf).T + np.abs(nA) @ np.abs(Wa).T
    u = EPS_BF16 * (1 + 2.0 ** -15)
    bound = u * Ssum + u * (np.abs(K) + u * Ssum) + 1e-15
    assert np.all(np.abs(Kb - K) <= bound)


def test_bf16_form_kernels_second_derivation():
    # the fold and both roundings written again with NumPy sums and torch's
    # BF16 conversion; the two FP64 sums differ only in order, which can move
    # an FP32 rounding at a tie, so a handful of one-step differences may show
    rng = np.random.default_rng(50)
    lvl = 2
    lab = _rng_labels((16, 16, 16), 51)
    img = oracle.avgpool2(oracle.image(lab))
    W = rng.uniform(-0.2, 0.2, (27, 3, 27))
    B = rng.uniform(-0.5, 0.5, 27)
    Fc = 8.0
    Wf = _torch_bf16((W[:, 0, :] - W[:, 2, :]) / Fc)
    Wa = _torch_bf16((W[:, 1, :] - W[:, 2, :]) / Fc)
    Bp = _torch_bf16(B + W[:, 2, :].sum(axis=1))
    nz, ny, nx = img.shape[1:]
    pf, pa = np.pad(img[0], 1), np.pad(img[1], 1)
    K = np.empty((nz, ny, nx, 27))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                f = Fc * pf[z:z + 3, y:y + 3, x:x + 3].ravel()
                a = Fc * pa[z:z + 3, y:y + 3, x:x + 3].ravel()
                K[z, y, x] = Bp + Wf @ f + Wa @ a
    K = _torch_bf16(K)
    Kb = oracle.cconv_kernels_bf16(img, W, B, lvl)
    diff = Kb != K
    assert diff.mean() < 1e-3
    np.testing.assert_allclose(Kb, K, rtol=2 * EPS_BF16, atol=0)


def test_bf16_form_network_is_linear_and_reduces_to_one_cconv():
    rng = np.random.default_rng(60)
    lab = _rng_labels((16, 16, 16), 61)
    w = synth.init_weights(3, 62, spread=0.05)
    r1, r2 = rng.standard_normal(lab.shape), rng.standard_normal(lab.shape)
    z12 = oracle.network(lab, 3, w, r1 + 2 * r2, form="bf16")
    z1, z2 = oracle.network(lab, 3, w, r1, form="bf16"), oracle.network(lab, 3, w, r2, form="bf16")
    np.testing.assert_allclose(z12, z1 + 2 * z2, atol=1e-11 * np.abs(z12).max())
    # the form changes the output by about the BF16 rounding, not more
    z = oracle.network(lab, 3, w, r1 + 2 * r2)
    e = np.linalg.norm(z12 - z) / np.linalg.norm(z)
    assert 1e-5 < e < 2e-2
    # L = 1: the network is the BF16 CConv of level 1 on the fluid-masked input, masked
    w1 = synth.init_weights(1, 63, spread=0.05)
    W, B = w1[: 27 * 3 * 27].reshape(27, 3, 27), w1[27 * 3 * 27:]
    v = np.where(lab == F, r1, 0.0)
    want = np.where(lab == F, oracle.cconv_bf16(oracle.image(lab), W, B, v, 1), 0.0)
    np.testing.assert_allclose(oracle.network(lab, 1, w1, r1, form="bf16"), want, rtol=0, atol=1e-13)


def test_bf16_form_solve_reaches_tolerance():
    lab = synth.pool_scene(32, 1000)
    rhs = synth.rhs_normal(lab, 1001)
    w = synth.init_weights(4, 7)
    r16 = oracle.npsdo(lab, rhs, L=4, w=w, tol=1e-6, max_iter=500, prec=oracle.PREC_NETWORK_BF16)
    r64 = oracle.npsdo(lab, rhs, L=4, w=w, tol=1e-6, max_iter=500)
    assert r16["status"] == oracle.OK and r16["relres"] < 1e-6
    assert abs(r16["iters"] - r64["iters"]) <= 3
    bm = np.where(lab == F, rhs, 0.0)
    assert np.linalg.norm(bm - oracle.lap_apply(lab, r16["x"])) / np.linalg.norm(bm) < 1e-6
