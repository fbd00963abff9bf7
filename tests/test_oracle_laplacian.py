"""Pins of the oracle's masked 7-point Laplacian (Sec. 3.1-3.2) against
closed-form eigenpairs and structural facts that the paper states.

A plausible mistake (wrong diagonal rule, a dropped neighbour, air counted as
fluid, grid exterior not treated as solid, non-empty non-fluid rows) breaks at
least one of these."""
import numpy as np
import pytest

import oracle
from paper_2310_00177_b300 import synth

S, F, A = 0, 1, 2


def _mesh(m):
    return np.meshgrid(np.arange(m[0]), np.arange(m[1]), np.arange(m[2]), indexing="ij")


def test_dirichlet_box_sine_modes():
    # fluid cube m^3 inside an air shell: every fluid cell has 6 fluid-or-air
    # neighbours, so A is the Dirichlet Laplacian with sine eigenvectors.
    m = 6
    lab = np.full((m + 2,) * 3, A, np.uint8)
    lab[1:-1, 1:-1, 1:-1] = F
    iz, iy, ix = _mesh((m, m, m))
    for k in [(1, 1, 1), (2, 1, 3), (6, 5, 4)]:
        v = np.zeros(lab.shape)
        mode = (np.sin(np.pi * k[0] * (iz + 1) / (m + 1)) * np.sin(np.pi * k[1] * (iy + 1) / (m + 1))
                * np.sin(np.pi * k[2] * (ix + 1) / (m + 1)))
        v[1:-1, 1:-1, 1:-1] = mode
        lam = sum(2 - 2 * np.cos(np.pi * kk / (m + 1)) for kk in k)
        np.testing.assert_allclose(oracle.lap_apply(lab, v), lam * v, atol=1e-12)


def test_neumann_box_cosine_modes_and_constant_nullspace():
    # an all-fluid grid: the exterior counts as solid, so A is the pure-Neumann
    # Laplacian with cell-centred cosine eigenvectors and constant null vector.
    m = (4, 5, 6)
    lab = np.full(m, F, np.uint8)
    iz, iy, ix = _mesh(m)
    for k in [(0, 0, 0), (1, 0, 0), (1, 2, 3), (3, 4, 5)]:
        v = (np.cos(np.pi * k[0] * (iz + 0.5) / m[0]) * np.cos(np.pi * k[1] * (iy + 0.5) / m[1])
             * np.cos(np.pi * k[2] * (ix + 0.5) / m[2]))
        lam = sum(2 - 2 * np.cos(np.pi * kk / mm) for kk, mm in zip(k, m))
        np.testing.assert_allclose(oracle.lap_apply(lab, v), lam * v, atol=1e-12)
    np.testing.assert_allclose(oracle.lap_apply(lab, np.ones(m)), 0.0, atol=1e-14)


def test_mixed_column_modes():
    # fluid block with solid walls/bottom (grid exterior) and an air layer on
    # top: Neumann in x, y and at the bottom, Dirichlet at the top.  The z
    # modes are cos(theta (i + 1/2)) with theta = (2k-1) pi / (2m+1).
    mz, my, mx = 7, 3, 4
    lab = np.full((mz + 1, my, mx), F, np.uint8)
    lab[mz] = A
    iz, iy, ix = _mesh((mz, my, mx))
    for kz, ky, kx in [(1, 0, 0), (2, 1, 3), (7, 2, 1)]:
        th = (2 * kz - 1) * np.pi / (2 * mz + 1)
        mode = np.cos(th * (iz + 0.5)) * np.cos(np.pi * ky * (iy + 0.5) / my) * np.cos(np.pi * kx * (ix + 0.5) / mx)
        v = np.zeros(lab.shape)
        v[:mz] = mode
        lam = (2 - 2 * np.cos(th)) + (2 - 2 * np.cos(np.pi * ky / my)) + (2 - 2 * np.cos(np.pi * kx / mx))
        np.testing.assert_allclose(oracle.lap_apply(lab, v), lam * v, atol=1e-12)


def _dense(lab):
    n = lab.size
    M = np.zeros((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        M[:, j] = oracle.lap_apply(lab, e.reshape(lab.shape)).ravel()
        e[j] = 0.0
    return M


def _random_labels(shape, seed, p=(0.25, 0.55, 0.2)):
    rng = np.random.default_rng(seed)
    return rng.choice(np.array([S, F, A], np.uint8), size=shape, p=p)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_symmetric_empty_nonfluid_rows_and_integer_stencil(seed):
    lab = _random_labels((5, 6, 7), seed)
    M = _dense(lab)
    np.testing.assert_array_equal(M, M.T)
    nonfluid = (lab != F).ravel()
    assert not M[nonfluid].any() and not M[:, nonfluid].any()
    # integer entries: off-diagonals -1 on fluid-fluid 6-neighbours, diagonal
    # in 0..6 equal to the count of fluid-or-air neighbours
    off = M - np.diag(np.diag(M))
    assert set(np.unique(off)) <= {0.0, -1.0}
    assert set(np.unique(np.diag(M))) <= set(float(k) for k in range(7))
    # a fluid row's sum equals its number of air neighbours (fluid ones
    # cancel, solid ones and the grid exterior are dropped)
    pad = np.pad(lab, 1, constant_values=S)
    nair = np.zeros(lab.shape)
    for ax in range(3):
        for sh in (-1, 1):
            nair += np.roll(pad, sh, axis=ax)[1:-1, 1:-1, 1:-1] == A
    fl = ~nonfluid
    np.testing.assert_array_equal(M[fl].sum(axis=1), nair.ravel()[fl])


@pytest.mark.parametrize("seed", [3, 4, 5, 6])
def test_nullspace_dimension_is_number_of_pure_neumann_components(seed):
    lab = _random_labels((5, 5, 6), seed, p=(0.35, 0.5, 0.15))
    fl = (lab == F).ravel()
    M = _dense(lab)[np.ix_(fl, fl)]
    ev = np.linalg.eigvalsh(M)
    assert ev.min() > -1e-10  # positive semi-definite
    _, pure = synth.neumann_components(lab)
    assert int(np.sum(ev < 1e-9)) == len(pure)


def test_positive_definite_when_every_component_touches_air():
    lab = synth.pool_scene(8, 3)
    _, pure = synth.neumann_components(lab)
    assert len(pure) == 0
    fl = (lab == F).ravel()
    M = _dense(lab)[np.ix_(fl, fl)]
    np.linalg.cholesky(M)  # raises if not positive definite
