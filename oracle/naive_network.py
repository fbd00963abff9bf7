"""Second, independent derivation of the network of Alg. 2 for tiny grids.

TEST INFRASTRUCTURE ONLY.  Written directly from the formulas of Sec. 4.2.1
with NumPy padding and per-cell Python loops (no code shared with
``npsdo_oracle.c``), so that the C oracle can be pinned against it on 8^3 and
16^3 inputs.  Slow by design: one Python iteration per cell.

Same conventions as the C oracle: image channels (fluid, air, solid), padding
of the image with solid pixels and of vectors with zeros, tap order
t = 9*(dz+1) + 3*(dy+1) + (dx+1).
"""
from __future__ import annotations

import numpy as np

FLUID, AIR, SOLID = 1, 2, 0


def onehot(labels):
    return np.stack([(labels == FLUID), (labels == AIR), (labels == SOLID)]).astype(np.float64)


def pool(f):
    """2x2x2 mean over the last three axes."""
    s = f.shape
    g = f.reshape(s[:-3] + (s[-3] // 2, 2, s[-2] // 2, 2, s[-1] // 2, 2))
    return g.mean(axis=(-5, -3, -1))


def _lin_up(a, axis):
    """Linear x2 upsampling along one axis, half-pixel centres, edge clamp."""
    n = a.shape[axis]
    f = np.arange(2 * n)
    src = np.maximum((f + 0.5) / 2.0 - 0.5, 0.0)
    i0 = np.minimum(np.floor(src).astype(int), n - 1)
    i1 = np.minimum(i0 + 1, n - 1)
    lam = src - i0
    a0 = np.take(a, i0, axis=axis)
    a1 = np.take(a, i1, axis=axis)
    shape = [1] * a.ndim
    shape[axis] = 2 * n
    lam = lam.reshape(shape)
    return a0 * (1 - lam) + a1 * lam


def interp(c):
    return _lin_up(_lin_up(_lin_up(c, 0), 1), 2)


def cconv(img, W, B, v):
    """out[p] = sum_a (B_a + sum_{c,l} W[a,c,l] I_c(p+l)) v(p+a)."""
    W = np.reshape(W, (27, 81))
    nz, ny, nx = v.shape
    ipad = np.pad(img, ((0, 0), (1, 1), (1, 1), (1, 1)))
    ipad[2, :, :, :] = np.pad(img[2], 1, constant_values=1.0)  # solid padding
    vpad = np.pad(v, 1)
    out = np.zeros_like(v)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                win_i = ipad[:, z:z + 3, y:y + 3, x:x + 3].reshape(3, 27)  # [c, l]
                K = W @ win_i.reshape(81) + B
                out[z, y, x] = K @ vpad[z:z + 3, y:y + 3, x:x + 3].reshape(27)
    return out


def aff(img, Wbar, Bbar):
    nz, ny, nx = img.shape[1:]
    ipad = np.pad(img, ((0, 0), (1, 1), (1, 1), (1, 1)))
    ipad[2] = np.pad(img[2], 1, constant_values=1.0)
    Wbar = np.reshape(Wbar, (3, 27))
    total = 0.0
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                total += float(np.sum(Wbar * ipad[:, z:z + 3, y:y + 3, x:x + 3].reshape(3, 27)))
    return Bbar + total / (27.0 * nz * ny * nx)


def network(labels, L, w, r):
    w = np.asarray(w, np.float64)
    C, A = 27 * 3 * 27 + 27, 82
    per = 2 * C + 2 * A

    def blk(o, size):
        return w[o:o + size]

    def conv_params(o):
        p = blk(o, C)
        return p[:2187], p[2187:]

    img = [None, onehot(labels)]
    r1 = [None, np.where(labels == FLUID, r, 0.0)]
    x1 = [None] * (L + 1)
    for lvl in range(1, L):
        img.append(pool(img[lvl]))
        Wc, Bc = conv_params((lvl - 1) * per)
        x1[lvl] = cconv(img[lvl], Wc, Bc, r1[lvl])
        r1.append(pool(x1[lvl]))
    Wc, Bc = conv_params((L - 1) * per)
    x = [None] * (L + 1)
    x[L] = cconv(img[L], Wc, Bc, r1[L])
    for lvl in range(L - 1, 0, -1):
        o = (lvl - 1) * per
        r2 = interp(x[lvl + 1])
        Wc, Bc = conv_params(o + C)
        x2 = cconv(img[lvl], Wc, Bc, r2)
        a1 = blk(o + 2 * C, A)
        a2 = blk(o + 2 * C + A, A)
        c1 = aff(img[lvl], a1[:81], a1[81])
        c2 = aff(img[lvl], a2[:81], a2[81])
        x[lvl] = c1 * x1[lvl] + c2 * x2
    return np.where(labels == FLUID, x[1], 0.0)
