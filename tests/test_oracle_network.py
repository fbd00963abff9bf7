"""Pins of the oracle's network pieces (Sec. 4.2.1, Alg. 2): CConv, Aff,
pooling, interpolation and the recursive network.

Pins are special cases that reduce to library routines (torch conv3d,
avg_pool3d, trilinear interpolate on the CPU), closed forms, the properties
the paper states (linearity in r, channels summing to one, any size divisible
by 2^(L-1)) and a second, independently written NumPy derivation."""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fn

import oracle
from oracle import naive_network
from paper_2310_00177_b300 import synth

S, F, A = 0, 1, 2


def _rng_labels(shape, seed, p=(0.3, 0.45, 0.25)):
    rng = np.random.default_rng(seed)
    return rng.choice(np.array([S, F, A], np.uint8), size=shape, p=p)


def _conv3d(v, k27):
    """Zero-padded 3x3x3 cross-correlation: out[p] = sum_a k[a] v[p + a]."""
    vt = torch.from_numpy(np.asarray(v, np.float64))[None, None]
    kt = torch.from_numpy(np.asarray(k27, np.float64).reshape(1, 1, 3, 3, 3))
    return Fn.conv3d(vt, kt, padding=1)[0, 0].numpy()


def test_cconv_with_zero_W_is_conv3d_with_bias_kernel():
    rng = np.random.default_rng(0)
    lab = _rng_labels((5, 6, 7), 1)
    img = oracle.image(lab)
    B = rng.standard_normal(27)
    v = rng.standard_normal(lab.shape)
    out = oracle.cconv(img, np.zeros((27, 3, 27)), B, v)
    np.testing.assert_allclose(out, _conv3d(v, B), atol=1e-13)


def test_cconv_all_solid_image_is_conv3d_everywhere():
    # an all-solid grid padded with solid: every window is all solid, so the
    # kernel is B + sum_l W[:, solid, l] at every cell, boundary included.
    rng = np.random.default_rng(2)
    lab = np.full((4, 5, 6), S, np.uint8)
    W = rng.standard_normal((27, 3, 27))
    B = rng.standard_normal(27)
    v = rng.standard_normal(lab.shape)
    out = oracle.cconv(oracle.image(lab), W, B, v)
    np.testing.assert_allclose(out, _conv3d(v, B + W[:, 2, :].sum(axis=1)), atol=1e-12)


def test_cconv_all_fluid_image_interior_is_conv3d():
    rng = np.random.default_rng(3)
    lab = np.full((6, 6, 7), F, np.uint8)
    W = rng.standard_normal((27, 3, 27))
    B = rng.standard_normal(27)
    v = rng.standard_normal(lab.shape)
    out = oracle.cconv(oracle.image(lab), W, B, v)
    ref = _conv3d(v, B + W[:, 0, :].sum(axis=1))
    np.testing.assert_allclose(out[1:-1, 1:-1, 1:-1], ref[1:-1, 1:-1, 1:-1], atol=1e-12)
    # a boundary cell sees solid padding on one side: its kernel picks up
    # W[:, solid, l] for the outside window entries instead
    K = oracle.cconv_kernels(oracle.image(lab), W, B)
    outside = [l for l in range(27) if l // 9 == 0]  # dz = -1 rows, outside at z = 0
    inside = [l for l in range(27) if l // 9 != 0]
    expect = B + W[:, 0, inside].sum(axis=1) + W[:, 2, outside].sum(axis=1)
    np.testing.assert_allclose(K[0, 3, 3], expect, atol=1e-12)


@pytest.mark.parametrize("a_star,c_star,l_star", [(0, 1, 5), (13, 0, 26), (22, 2, 9)])
def test_kernel_generator_orientation_single_entry(a_star, c_star, l_star):
    # W has one non-zero entry W[a*, c*, l*] = 1 and B = 0; with a single cell q
    # of the channel c* inside a grid of another material, K_a(p) is 1 exactly
    # for a = a* and p + l* = q (and the padding contributes for c* = solid).
    lab = np.full((5, 5, 5), F if c_star != 0 else A, np.uint8)
    q = (2, 1, 3)
    lab[q] = [F, A, S][c_star]
    W = np.zeros((27, 3, 27))
    W[a_star, c_star, l_star] = 1.0
    K = oracle.cconv_kernels(oracle.image(lab), W, np.zeros(27))
    dz, dy, dx = l_star // 9 - 1, (l_star // 3) % 3 - 1, l_star % 3 - 1
    expect = np.zeros((5, 5, 5, 27))
    for z in range(5):
        for y in range(5):
            for x in range(5):
                pz, py, px = z + dz, y + dy, x + dx
                outside = not (0 <= pz < 5 and 0 <= py < 5 and 0 <= px < 5)
                if (pz, py, px) == q or (outside and c_star == 2):
                    expect[z, y, x, a_star] = 1.0
    np.testing.assert_array_equal(K, expect)


def test_avgpool_matches_torch():
    rng = np.random.default_rng(4)
    f = rng.standard_normal((3, 6, 4, 8))
    ref = Fn.avg_pool3d(torch.from_numpy(f)[None], 2)[0].numpy()
    np.testing.assert_allclose(oracle.avgpool2(f), ref, atol=1e-14)


def test_interp_matches_torch_trilinear_half_pixel():
    rng = np.random.default_rng(5)
    c = rng.standard_normal((3, 4, 5))
    ref = Fn.interpolate(torch.from_numpy(c)[None, None], scale_factor=2, mode="trilinear",
                         align_corners=False)[0, 0].numpy()
    np.testing.assert_allclose(oracle.interp_up2(c), ref, atol=1e-13)


def test_pool_and_interp_adjoints():
    rng = np.random.default_rng(6)
    u = rng.standard_normal((4, 6, 8))
    g = rng.standard_normal((2, 3, 4))
    assert abs(np.vdot(oracle.avgpool2(u), g) - np.vdot(u, oracle.avgpool2_adjoint(g))) < 1e-12
    gf = rng.standard_normal((4, 6, 8))
    assert abs(np.vdot(oracle.interp_up2(g), gf) - np.vdot(g, oracle.interp_up2_adjoint(gf))) < 1e-12


def test_aff_closed_forms():
    rng = np.random.default_rng(7)
    Wb = rng.standard_normal((3, 27))
    # Wbar = 0 gives the bias
    lab = _rng_labels((4, 4, 6), 8)
    assert oracle.aff(oracle.image(lab), np.zeros((3, 27)), 0.7) == pytest.approx(0.7, abs=1e-15)
    # all solid: every window entry is solid
    sol = np.full((4, 4, 6), S, np.uint8)
    assert oracle.aff(oracle.image(sol), Wb, 0.3) == pytest.approx(0.3 + Wb[2].sum() / 27.0, rel=1e-13)
    # all fluid: for offset l, prod_d (n_d - |l_d|) cells see fluid, the rest solid padding
    m = (4, 5, 6)
    flu = np.full(m, F, np.uint8)
    n = np.prod(m)
    total = 0.0
    for l in range(27):
        d = (abs(l // 9 - 1), abs((l // 3) % 3 - 1), abs(l % 3 - 1))
        cnt = (m[0] - d[0]) * (m[1] - d[1]) * (m[2] - d[2])
        total += Wb[0, l] * cnt + Wb[2, l] * (n - cnt)
    assert oracle.aff(oracle.image(flu), Wb, -0.2) == pytest.approx(-0.2 + total / (27 * n), rel=1e-12)


def test_pyramid_channels_sum_to_one():
    lab = _rng_labels((16, 16, 16), 9)
    img = oracle.image(lab)
    for _ in range(4):
        np.testing.assert_allclose(img.sum(axis=0), 1.0, atol=1e-15)
        img = oracle.avgpool2(img)


def test_weight_counts():
    assert oracle.weight_count(4) == 15990
    assert oracle.weight_count(6) == 25174
    assert synth.weight_count(4) == oracle.weight_count(4)


@pytest.mark.parametrize("shape,L,seed", [((8, 8, 8), 4, 10), ((8, 8, 16), 3, 11), ((4, 8, 8), 2, 12)])
def test_network_matches_independent_numpy_derivation(shape, L, seed):
    rng = np.random.default_rng(seed)
    lab = _rng_labels(shape, seed)
    w = rng.standard_normal(oracle.weight_count(L)) * 0.3
    r = rng.standard_normal(shape)
    z = oracle.network(lab, L, w, r)
    zn = naive_network.network(lab, L, w, r)
    np.testing.assert_allclose(z, zn, rtol=1e-11, atol=1e-11 * np.abs(zn).max())


def test_network_is_linear_in_r():
    rng = np.random.default_rng(13)
    lab = _rng_labels((8, 8, 8), 13)
    w = rng.standard_normal(oracle.weight_count(4)) * 0.3
    r, s = rng.standard_normal((2, 8, 8, 8))
    lhs = oracle.network(lab, 4, w, 2.5 * r - 0.75 * s)
    rhs = 2.5 * oracle.network(lab, 4, w, r) - 0.75 * oracle.network(lab, 4, w, s)
    np.testing.assert_allclose(lhs, rhs, atol=1e-10 * np.abs(rhs).max())


def _identity_weights(L, aff1, aff2):
    w = np.zeros(oracle.weight_count(L))
    per = 2 * oracle.CCONV_PARAMS + 2 * oracle.AFF_PARAMS
    for lvl in range(1, L + 1):
        o = (lvl - 1) * per
        w[o + 2187 + 13] = 1.0
        if lvl < L:
            w[o + oracle.CCONV_PARAMS + 2187 + 13] = 1.0
            w[o + 2 * oracle.CCONV_PARAMS + 81] = aff1
            w[o + 2 * oracle.CCONV_PARAMS + oracle.AFF_PARAMS + 81] = aff2
    return w


def test_network_structure_with_identity_convolutions():
    # CConv = identity (W = 0, B = centre tap): with Aff1 = 1, Aff2 = 0 the
    # network is the masked identity; with Aff1 = 0, Aff2 = 1 it is
    # interp^(L-1)(pool^(L-1)(r)), masked.
    rng = np.random.default_rng(14)
    lab = _rng_labels((16, 16, 8), 14)
    r = rng.standard_normal(lab.shape)
    rm = np.where(lab == F, r, 0.0)
    L = 4
    z = oracle.network(lab, L, _identity_weights(L, 1.0, 0.0), r)
    np.testing.assert_allclose(z, rm, atol=1e-14)
    z = oracle.network(lab, L, _identity_weights(L, 0.0, 1.0), r)
    t = torch.from_numpy(rm)[None, None]
    for _ in range(L - 1):
        t = Fn.avg_pool3d(t, 2)
    for _ in range(L - 1):
        t = Fn.interpolate(t, scale_factor=2, mode="trilinear", align_corners=False)
    np.testing.assert_allclose(z, np.where(lab == F, t[0, 0].numpy(), 0.0), atol=1e-13)


def test_single_level_network_is_one_cconv():
    rng = np.random.default_rng(15)
    lab = _rng_labels((5, 6, 7), 15)
    w = rng.standard_normal(oracle.weight_count(1))
    r = rng.standard_normal(lab.shape)
    rm = np.where(lab == F, r, 0.0)
    ref = oracle.cconv(oracle.image(lab), w[:2187], w[2187:], rm)
    np.testing.assert_allclose(oracle.network(lab, 1, w, r), np.where(lab == F, ref, 0.0), atol=1e-13)


def test_sizes_not_divisible_by_2_pow_L_minus_1_are_rejected():
    lab = np.full((8, 8, 12), F, np.uint8)
    with pytest.raises(ValueError):
        oracle.network(lab, 4, np.zeros(oracle.weight_count(4)), np.zeros(lab.shape))
    oracle.network(lab, 3, np.zeros(oracle.weight_count(3)), np.zeros(lab.shape))
