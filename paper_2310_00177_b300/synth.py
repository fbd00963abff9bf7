"""Seeded synthetic inputs shaped like the paper's fluid scenes.

This module only draws random numbers and rasterises shapes; it holds none of
the solver's or the network's arithmetic, so both the CUDA path (tests, bench)
and the CPU oracle use it for their inputs.

The paper's own scenes (smoke around solids, scooping, water flowing around a
torus or ball, dam breaks; Sec. 5 and Table 3, grids of 128^3, 256x128^2 and
256^3) are not available, so seeded stand-ins with the same ingredients are
generated here: a solid outer shell (Neumann walls), solid spheres and boxes,
an air region above a free surface (Dirichlet), fluid elsewhere.

Label codes: 0 solid, 1 fluid, 2 air.  Arrays are (nz, ny, nx), x fastest, z up.
"""
from __future__ import annotations

import math

import numpy as np

SOLID, FLUID, AIR = 0, 1, 2

CCONV_PARAMS = 27 * 3 * 27 + 27
AFF_PARAMS = 3 * 27 + 1


def _grid(n):
    nz, ny, nx = n
    z = np.arange(nz, dtype=np.float32)[:, None, None]
    y = np.arange(ny, dtype=np.float32)[None, :, None]
    x = np.arange(nx, dtype=np.float32)[None, None, :]
    return z, y, x


def _stamp_sphere(solid, c, r):
    nz, ny, nx = solid.shape
    cz, cy, cx = c
    z0, z1 = max(0, int(math.floor(cz - r))), min(nz, int(math.ceil(cz + r)) + 1)
    y0, y1 = max(0, int(math.floor(cy - r))), min(ny, int(math.ceil(cy + r)) + 1)
    x0, x1 = max(0, int(math.floor(cx - r))), min(nx, int(math.ceil(cx + r)) + 1)
    if z0 >= z1 or y0 >= y1 or x0 >= x1:
        return
    z = np.arange(z0, z1, dtype=np.float32)[:, None, None] + 0.5
    y = np.arange(y0, y1, dtype=np.float32)[None, :, None] + 0.5
    x = np.arange(x0, x1, dtype=np.float32)[None, None, :] + 0.5
    m = (z - cz) ** 2 + (y - cy) ** 2 + (x - cx) ** 2 <= r * r
    solid[z0:z1, y0:y1, x0:x1] |= m


def _stamp_box(solid, c, h):
    nz, ny, nx = solid.shape
    cz, cy, cx = c
    hz, hy, hx = h
    z0, z1 = max(0, int(round(cz - hz))), min(nz, int(round(cz + hz)))
    y0, y1 = max(0, int(round(cy - hy))), min(ny, int(round(cy + hy)))
    x0, x1 = max(0, int(round(cx - hx))), min(nx, int(round(cx + hx)))
    if z0 < z1 and y0 < y1 and x0 < x1:
        solid[z0:z1, y0:y1, x0:x1] = True


def _shell(shape):
    s = np.zeros(shape, dtype=bool)
    s[0, :, :] = s[-1, :, :] = True
    s[:, 0, :] = s[:, -1, :] = True
    s[:, :, 0] = s[:, :, -1] = True
    return s


def pool_scene(n=32, seed=1000):
    """Small scene: solid shell, 3 solid spheres of radius U[3,6] with centres
    U[8,24]^3 (scaled by n/32), air above a flat free surface at z = 24 n/32."""
    rng = np.random.default_rng(seed)
    s = n / 32.0
    shape = (n, n, n)
    solid = _shell(shape)
    for _ in range(3):
        r = rng.uniform(3.0, 6.0) * s
        c = rng.uniform(8.0 * s, 24.0 * s, size=3)
        _stamp_sphere(solid, c, r)
    z, _, _ = _grid(shape)
    air = np.broadcast_to(z >= 24.0 * s, shape) & ~solid
    lab = np.full(shape, FLUID, np.uint8)
    lab[air] = AIR
    lab[solid] = SOLID
    return lab


def slosh_scene(n=128, seed=2000, frame=0, shape=None):
    """Scene shaped like the paper's mixed-BC examples at any size.

    Solid shell; K ~ U{10..40} solids, each a sphere (radius U[4,16] s) or an
    axis-aligned box (half extents U[4,16] s) with probability 1/2, s = n/128;
    free surface z_s(x, y) = 80 s + 8 sin(2 pi x/n + phi1) cos(2 pi y/n + phi2)
    with air above it.  ``frame`` animates the scene: solids translate +1 cell
    per frame along x (periodically) and both surface phases advance 0.2 rad.
    ``shape`` (nz, ny, nx) overrides the cube n^3 (s is then nz/128).
    """
    if shape is None:
        shape = (n, n, n)
    nz, ny, nx = shape
    s = nz / 128.0
    rng = np.random.default_rng(seed)
    K = int(rng.integers(10, 41))
    solid = _shell(shape)
    for _ in range(K):
        kind = rng.integers(0, 2)
        c = rng.uniform(0.0, 1.0, size=3) * np.array([nz, ny, nx], np.float64)
        c[2] = (c[2] + frame) % nx
        if kind == 0:
            _stamp_sphere(solid, c, rng.uniform(4.0, 16.0) * s)
        else:
            _stamp_box(solid, c, rng.uniform(4.0, 16.0, size=3) * s)
    phi1, phi2 = rng.uniform(0.0, 2.0 * math.pi, size=2) + 0.2 * frame
    z, y, x = _grid(shape)
    zs = 80.0 * s + 8.0 * np.sin(2 * math.pi * x / nx + phi1) * np.cos(2 * math.pi * y / ny + phi2)
    air = (z >= zs) & ~solid
    lab = np.full(shape, FLUID, np.uint8)
    lab[air] = AIR
    lab[solid] = SOLID
    return lab


def neumann_components(labels):
    """Connected fluid components (6-connectivity) that touch no air cell.

    Returns (component_id array, list of ids that are pure-Neumann)."""
    from scipy import ndimage

    fluid = labels == FLUID
    air = labels == AIR
    struct = ndimage.generate_binary_structure(3, 1)
    comp, ncomp = ndimage.label(fluid, structure=struct)
    near_air = ndimage.binary_dilation(air, structure=struct) & fluid
    touched = np.unique(comp[near_air])
    pure = np.setdiff1d(np.arange(1, ncomp + 1), touched)
    return comp, pure


def project_neumann(labels, b):
    """Zero b off fluid and remove its mean on every pure-Neumann component,
    so that the singular (constant-null-space) blocks are consistent."""
    b = np.where(labels == FLUID, b, 0.0)
    comp, pure = neumann_components(labels)
    if len(pure):
        sums = np.bincount(comp.ravel(), weights=b.ravel(), minlength=comp.max() + 1)
        cnts = np.bincount(comp.ravel(), minlength=comp.max() + 1)
        mean = np.zeros_like(sums)
        mean[pure] = sums[pure] / np.maximum(cnts[pure], 1)
        b = b - mean[comp] * (comp > 0)
    return b


def rhs_normal(labels, seed, dtype=np.float64):
    """b ~ N(0, 1) on fluid cells, zero elsewhere, projected per pure-Neumann
    component."""
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(labels.shape)
    return project_neumann(labels, b).astype(dtype)


def weight_count(L):
    return (L - 1) * (2 * CCONV_PARAMS + 2 * AFF_PARAMS) + CCONV_PARAMS


def init_weights(L=4, seed=0, spread=1.0 / 81.0, omega=1.0, level_gain=4.0):
    """Seeded random initial network weights (the paper does not state its
    initialisation).

    Every W, B, Wbar, Bbar entry is drawn from U(-spread, spread) and then a
    fixed multilevel starting point is added, so that the untrained network is
    already a usable preconditioner (about an additive multilevel smoother):
    the centre-tap bias B_13 of every CConv1/CConv2 block below the coarsest
    level gets +1, the coarsest CConv1 gets +omega*level_gain^(L-1)/6, Aff1 of
    level l gets Bbar += omega*level_gain^(l-1)/6 and Aff2 gets Bbar += 1.

    Layout: for level 1..L-1: CConv1 (W 27x3x27, B 27), CConv2, Aff1 (Wbar
    3x27, Bbar), Aff2; then CConv1 of level L."""
    rng = np.random.default_rng(seed)
    w = rng.uniform(-spread, spread, size=weight_count(L))
    per = 2 * CCONV_PARAMS + 2 * AFF_PARAMS
    centre = 27 * 3 * 27 + 13
    for lvl in range(1, L + 1):
        o = (lvl - 1) * per
        if lvl == L:
            w[o + centre] += omega * level_gain ** (lvl - 1) / 6.0
        else:
            w[o + centre] += 1.0
            w[o + CCONV_PARAMS + centre] += 1.0
            w[o + 2 * CCONV_PARAMS + 81] += omega * level_gain ** (lvl - 1) / 6.0
            w[o + 2 * CCONV_PARAMS + AFF_PARAMS + 81] += 1.0
    return w


def serving_requests(count=512, rate=200.0, sizes=(64, 128, 192, 256), seed=5000):
    """Poisson arrivals (exponential inter-arrival times, mean 1/rate s) of solve
    requests; each is frame f of an evolving scene of a size drawn uniformly
    from ``sizes``.  Returns a list of dicts (t_arrival, n, frame, scene_seed,
    rhs_seed)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    ns = rng.choice(np.asarray(sizes), size=count)
    frame_of = {}
    out = []
    for i in range(count):
        n = int(ns[i])
        f = frame_of.get(n, 0)
        frame_of[n] = f + 1
        out.append({"t_arrival": float(t[i]), "n": n, "frame": f, "scene_seed": seed + n,
                    "rhs_seed": seed * 7 + i})
    return out
