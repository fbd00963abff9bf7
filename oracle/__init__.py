"""FP64 CPU oracle for the NPSDO solve of arXiv 2310.00177 -- test infrastructure.

This package is the slow, literal reference implementation that the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
``paper_2310_00177_b300`` (the product) and never imports it, except for the
seeded input generators in ``paper_2310_00177_b300.synth``, which hold none of
the method's arithmetic.

Contents (each wraps a C function of ``npsdo_oracle.c``):

* ``lap_apply``          masked 7-point Laplacian (Sec. 3.2)
* ``image``, ``avgpool2``, ``interp_up2`` image pyramid / pooling /
  interpolation of Alg. 2
* ``cconv``, ``cconv_kernels``, ``cconv_backward``  CConv block (Sec. 4.2.1)
* ``round_bf16``, ``cconv_bf16``, ``cconv_kernels_bf16``  the CUDA library's
  BF16 form of CConv (kernel values rounded to BF16; a numerical form of the
  library, not of the paper), used by ``network(form="bf16")`` and by the
  solvers with ``prec=PREC_NETWORK_BF16``
* ``aff``, ``aff_grad``  Aff block (Sec. 4.2.1)
* ``network``, ``network_level``, ``network_backward`` Alg. 2 and its reverse
* ``loss``               training loss of Sec. 4.2.3 and its weight gradient
* ``npsdo``              Alg. 1
* ``npcg``               PCG / flexible PCG with the network as preconditioner
                         (Sec. 4.1, the appendix's solver variants)
* ``jacobi_pcg``         textbook Jacobi-preconditioned CG
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "npsdo_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

LAB_SOLID, LAB_FLUID, LAB_AIR = 0, 1, 2
CCONV_PARAMS = 27 * 3 * 27 + 27
AFF_PARAMS = 3 * 27 + 1

OK, BAD_ARG, BAD_DIMS, BAD_LABELS, NO_CONVERGENCE, BREAKDOWN = 0, 1, 2, 3, 4, 5

PREC_NETWORK, PREC_IDENTITY, PREC_DENSE, PREC_NETWORK_SYM, PREC_NETWORK_BF16 = 0, 1, 2, 3, 4
_NET_PRECS = (PREC_NETWORK, PREC_NETWORK_SYM, PREC_NETWORK_BF16)


def build(force: bool = False) -> str:
    """Compile ``npsdo_oracle.c`` into ``liboracle.so`` with gcc (no -ffast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        )
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i = ctypes.c_int


def _declare(L):
    L.or_lap_apply.argtypes = [_u8p, _i, _i, _i, _dp, _dp]
    L.or_lap_diag.argtypes = [_u8p, _i, _i, _i, _dp]
    L.or_image_from_labels.argtypes = [_u8p, _i, _i, _i, _dp]
    L.or_avgpool2.argtypes = [_dp, _i, _i, _i, _i, _dp]
    L.or_avgpool2_adjoint.argtypes = [_dp, _i, _i, _i, _dp]
    L.or_interp_up2.argtypes = [_dp, _i, _i, _i, _dp]
    L.or_interp_up2_adjoint.argtypes = [_dp, _i, _i, _i, _dp]
    L.or_cconv.argtypes = [_dp, _i, _i, _i, _dp, _dp, _dp, _dp]
    L.or_cconv_kernels.argtypes = [_dp, _i, _i, _i, _dp, _dp, _dp]
    L.or_cconv_backward.argtypes = [_dp, _i, _i, _i, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.or_aff.argtypes = [_dp, _i, _i, _i, _dp, ctypes.c_double]
    L.or_aff.restype = ctypes.c_double
    L.or_aff_grad.argtypes = [_dp, _i, _i, _i, _dp]
    L.or_weight_count.argtypes = [_i]
    L.or_weight_count.restype = ctypes.c_size_t
    L.or_network.argtypes = [_u8p, _i, _i, _i, _i, _dp, _dp, _dp]
    L.or_network_level.argtypes = [_u8p, _i, _i, _i, _i, _dp, _dp, _i, _i, _dp, _dp]
    L.or_network_backward.argtypes = [_u8p, _i, _i, _i, _i, _dp, _dp, _dp, _dp, _dp]
    L.or_loss.argtypes = [_u8p, _i, _i, _i, _i, _dp, _dp, _dp, _dp]
    L.or_npsdo.argtypes = [_u8p, _i, _i, _i, _i, _dp, _i, _dp, _dp, ctypes.c_double, _i, _i, _i,
                           _dp, ctypes.POINTER(_i), _dp, _dp]
    L.or_jacobi_pcg.argtypes = [_u8p, _i, _i, _i, _dp, ctypes.c_double, _i, _dp,
                                ctypes.POINTER(_i), _dp, _dp]
    L.or_npcg.argtypes = [_u8p, _i, _i, _i, _i, _dp, _i, _dp, _dp, ctypes.c_double, _i, _i, _i,
                          _dp, ctypes.POINTER(_i), _dp, _dp]
    L.or_check_labels.argtypes = [_u8p, _i, _i, _i]
    L.or_round_bf16.argtypes = [ctypes.c_double]
    L.or_round_bf16.restype = ctypes.c_double
    L.or_cconv_bf16.argtypes = [_dp, _i, _i, _i, _dp, _dp, _i, _dp, _dp]
    L.or_cconv_kernels_bf16.argtypes = [_dp, _i, _i, _i, _dp, _dp, _i, _dp]
    L.or_network_form.argtypes = [_u8p, _i, _i, _i, _i, _dp, _i, _dp, _dp]


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _lab(labels):
    labels = np.ascontiguousarray(labels, dtype=np.uint8)
    assert labels.ndim == 3
    nz, ny, nx = labels.shape
    return labels, labels.ctypes.data_as(_u8p), nx, ny, nz


def _null():
    return ctypes.cast(None, _dp)


def weight_count(L: int) -> int:
    return int(lib().or_weight_count(L))


def lap_apply(labels, d):
    labels, lp, nx, ny, nz = _lab(labels)
    d, dp = _f64(d)
    q = np.empty_like(d)
    lib().or_lap_apply(lp, nx, ny, nz, dp, q.ctypes.data_as(_dp))
    return q


def lap_diag(labels):
    labels, lp, nx, ny, nz = _lab(labels)
    out = np.empty(labels.shape, np.float64)
    lib().or_lap_diag(lp, nx, ny, nz, out.ctypes.data_as(_dp))
    return out


def image(labels):
    """Level-1 image, shape (3, nz, ny, nx), channels (fluid, air, solid)."""
    labels, lp, nx, ny, nz = _lab(labels)
    out = np.empty((3,) + labels.shape, np.float64)
    lib().or_image_from_labels(lp, nx, ny, nz, out.ctypes.data_as(_dp))
    return out


def avgpool2(field):
    """2x2x2 mean of a (C, nz, ny, nx) or (nz, ny, nx) field."""
    f = np.asarray(field, np.float64)
    squeeze = f.ndim == 3
    if squeeze:
        f = f[None]
    C, nz, ny, nx = f.shape
    f, fp = _f64(f)
    out = np.empty((C, nz // 2, ny // 2, nx // 2), np.float64)
    lib().or_avgpool2(fp, C, nx, ny, nz, out.ctypes.data_as(_dp))
    return out[0] if squeeze else out


def avgpool2_adjoint(gc):
    gc, gp = _f64(gc)
    cz, cy, cx = gc.shape
    out = np.empty((2 * cz, 2 * cy, 2 * cx), np.float64)
    lib().or_avgpool2_adjoint(gp, 2 * cx, 2 * cy, 2 * cz, out.ctypes.data_as(_dp))
    return out


def interp_up2(coarse):
    coarse, cp = _f64(coarse)
    cz, cy, cx = coarse.shape
    out = np.empty((2 * cz, 2 * cy, 2 * cx), np.float64)
    lib().or_interp_up2(cp, cx, cy, cz, out.ctypes.data_as(_dp))
    return out


def interp_up2_adjoint(gfine):
    gfine, gp = _f64(gfine)
    fz, fy, fx = gfine.shape
    out = np.empty((fz // 2, fy // 2, fx // 2), np.float64)
    lib().or_interp_up2_adjoint(gp, fx // 2, fy // 2, fz // 2, out.ctypes.data_as(_dp))
    return out


def _split_cconv(wb):
    wb = np.ascontiguousarray(wb, np.float64).ravel()
    assert wb.size == CCONV_PARAMS
    return wb[: 27 * 3 * 27].copy(), wb[27 * 3 * 27:].copy()


def cconv(img, W, B, v):
    """CConv of Sec. 4.2.1.  img (3,nz,ny,nx); W (27,3,27); B (27,); v (nz,ny,nx)."""
    img, ip = _f64(img)
    _, nz, ny, nx = img.shape
    W, wp = _f64(np.reshape(W, (27, 3, 27)))
    B, bp = _f64(np.reshape(B, (27,)))
    v, vp = _f64(v)
    out = np.empty((nz, ny, nx), np.float64)
    lib().or_cconv(ip, nx, ny, nz, wp, bp, vp, out.ctypes.data_as(_dp))
    return out


def cconv_kernels(img, W, B):
    img, ip = _f64(img)
    _, nz, ny, nx = img.shape
    W, wp = _f64(np.reshape(W, (27, 3, 27)))
    B, bp = _f64(np.reshape(B, (27,)))
    out = np.empty((nz, ny, nx, 27), np.float64)
    lib().or_cconv_kernels(ip, nx, ny, nz, wp, bp, out.ctypes.data_as(_dp))
    return out


def cconv_backward(img, W, B, v, g):
    img, ip = _f64(img)
    _, nz, ny, nx = img.shape
    W, wp = _f64(np.reshape(W, (27, 3, 27)))
    B, bp = _f64(np.reshape(B, (27,)))
    v, vp = _f64(v)
    g, gp = _f64(g)
    gv = np.zeros((nz, ny, nx))
    gW = np.zeros((27, 3, 27))
    gB = np.zeros(27)
    lib().or_cconv_backward(ip, nx, ny, nz, wp, bp, vp, gp, gv.ctypes.data_as(_dp),
                            gW.ctypes.data_as(_dp), gB.ctypes.data_as(_dp))
    return gv, gW, gB


def aff(img, Wbar, Bbar):
    img, ip = _f64(img)
    _, nz, ny, nx = img.shape
    Wbar, wp = _f64(np.reshape(Wbar, (3, 27)))
    return float(lib().or_aff(ip, nx, ny, nz, wp, float(Bbar)))


def aff_grad(img):
    img, ip = _f64(img)
    _, nz, ny, nx = img.shape
    out = np.empty((3, 27))
    lib().or_aff_grad(ip, nx, ny, nz, out.ctypes.data_as(_dp))
    return out


def _check(st):
    if st not in (OK, NO_CONVERGENCE):
        raise ValueError(f"oracle status {st}")
    return st


def network(labels, L, w, r, form="fp64"):
    """z = P_net(I, r) (Alg. 2), output restricted to fluid; form="bf16" gives
    the library's BF16 form (every CConv kernel value rounded to BF16)."""
    labels, lp, nx, ny, nz = _lab(labels)
    w, wp = _f64(w)
    assert w.size == weight_count(L)
    r, rp = _f64(r)
    z = np.empty(labels.shape, np.float64)
    if form == "fp64":
        _check(lib().or_network(lp, nx, ny, nz, L, wp, rp, z.ctypes.data_as(_dp)))
    else:
        assert form == "bf16"
        _check(lib().or_network_form(lp, nx, ny, nz, L, wp, 1, rp, z.ctypes.data_as(_dp)))
    return z


def round_bf16(v):
    """Nearest BF16 value (ties to even) of the FP32 rounding of each entry."""
    f = lib().or_round_bf16
    return np.vectorize(lambda t: f(float(t)), otypes=[np.float64])(np.asarray(v, np.float64))


def cconv_bf16(img, W, B, v, lvl):
    """The BF16-form CConv of a level-``lvl`` field (fold by the channel-sum
    identity, round the folded weights and every kernel value to BF16)."""
    img, ip = _f64(img)
    _, nz, ny, nx = img.shape
    W, wp = _f64(np.reshape(W, (27, 3, 27)))
    B, bp = _f64(np.reshape(B, (27,)))
    v, vp = _f64(v)
    out = np.empty((nz, ny, nx))
    lib().or_cconv_bf16(ip, nx, ny, nz, wp, bp, int(lvl), vp, out.ctypes.data_as(_dp))
    return out


def cconv_kernels_bf16(img, W, B, lvl):
    """BF16-form per-cell kernels K[z, y, x, a] of a level-``lvl`` image."""
    img, ip = _f64(img)
    _, nz, ny, nx = img.shape
    W, wp = _f64(np.reshape(W, (27, 3, 27)))
    B, bp = _f64(np.reshape(B, (27,)))
    K = np.empty((nz, ny, nx, 27))
    lib().or_cconv_kernels_bf16(ip, nx, ny, nz, wp, bp, int(lvl), K.ctypes.data_as(_dp))
    return K


WHICH = {"x1": 0, "r2": 1, "x2": 2, "x": 3, "r1": 4}


def network_level(labels, L, w, r, lvl, which):
    """An intermediate of one forward pass at level ``lvl``; returns (field, (c1, c2))."""
    labels, lp, nx, ny, nz = _lab(labels)
    w, wp = _f64(w)
    r, rp = _f64(r)
    s = 1 << (lvl - 1)
    out = np.empty((nz // s, ny // s, nx // s), np.float64)
    c12 = np.zeros(2)
    _check(lib().or_network_level(lp, nx, ny, nz, L, wp, rp, lvl, WHICH[which],
                                  out.ctypes.data_as(_dp), c12.ctypes.data_as(_dp)))
    return out, (float(c12[0]), float(c12[1]))


def network_backward(labels, L, w, r, gz):
    labels, lp, nx, ny, nz = _lab(labels)
    w, wp = _f64(w)
    r, rp = _f64(r)
    gz, gzp = _f64(gz)
    gw = np.zeros(w.size)
    gr = np.zeros(labels.shape)
    _check(lib().or_network_backward(lp, nx, ny, nz, L, wp, rp, gzp, gw.ctypes.data_as(_dp),
                                     gr.ctypes.data_as(_dp)))
    return gw, gr


def loss(labels, L, w, b, grad=True):
    """Loss = ||b - A P_net(I, b)||_2 and (optionally) its weight gradient."""
    labels, lp, nx, ny, nz = _lab(labels)
    w, wp = _f64(w)
    b, bp = _f64(b)
    out = ctypes.c_double(0.0)
    gw = np.zeros(w.size) if grad else None
    _check(lib().or_loss(lp, nx, ny, nz, L, wp, bp, ctypes.byref(out),
                         gw.ctypes.data_as(_dp) if grad else _null()))
    return (out.value, gw) if grad else out.value


def npsdo(labels, b, *, L=4, w=None, tol=1e-6, max_iter=1000, n_ortho=2, residual_mode=0,
          prec=PREC_NETWORK, pdense=None):
    """Alg. 1.  Returns dict(x, iters, status, res_hist, relres)."""
    labels, lp, nx, ny, nz = _lab(labels)
    n = labels.size
    if prec in _NET_PRECS:
        w, wp = _f64(w)
        assert w.size == weight_count(L)
    else:
        wp = _null()
    if prec == PREC_DENSE:
        pdense, pdp = _f64(pdense)
        assert pdense.shape == (n, n)
    else:
        pdp = _null()
    b, bp = _f64(b)
    x = np.zeros(labels.shape)
    it = ctypes.c_int(0)
    hist = np.zeros(max_iter + 1)
    relres = ctypes.c_double(0.0)
    st = lib().or_npsdo(lp, nx, ny, nz, L, wp, prec, pdp, bp, float(tol), int(max_iter), int(n_ortho),
                        int(residual_mode), x.ctypes.data_as(_dp), ctypes.byref(it),
                        hist.ctypes.data_as(_dp), ctypes.byref(relres))
    if st not in (OK, NO_CONVERGENCE, BREAKDOWN):
        raise ValueError(f"oracle status {st}")
    return {"x": x, "iters": it.value, "status": st, "res_hist": hist[: it.value + 1].copy(),
            "relres": relres.value}


def npcg(labels, b, *, L=4, w=None, tol=1e-6, max_iter=1000, flexible=False, residual_mode=0,
         prec=PREC_NETWORK, pdense=None):
    """PCG (flexible=False) or flexible PCG (flexible=True) with the network
    as preconditioner (Sec. 4.1; the appendix's solver-variant comparison).
    Returns dict(x, iters, status, res_hist, relres) as npsdo does."""
    labels, lp, nx, ny, nz = _lab(labels)
    n = labels.size
    if prec in _NET_PRECS:
        w, wp = _f64(w)
        assert w.size == weight_count(L)
    else:
        wp = _null()
    if prec == PREC_DENSE:
        pdense, pdp = _f64(pdense)
        assert pdense.shape == (n, n)
    else:
        pdp = _null()
    b, bp = _f64(b)
    x = np.zeros(labels.shape)
    it = ctypes.c_int(0)
    hist = np.zeros(max_iter + 1)
    relres = ctypes.c_double(0.0)
    st = lib().or_npcg(lp, nx, ny, nz, L, wp, prec, pdp, bp, float(tol), int(max_iter), int(bool(flexible)),
                       int(residual_mode), x.ctypes.data_as(_dp), ctypes.byref(it),
                       hist.ctypes.data_as(_dp), ctypes.byref(relres))
    if st not in (OK, NO_CONVERGENCE, BREAKDOWN):
        raise ValueError(f"oracle status {st}")
    return {"x": x, "iters": it.value, "status": st, "res_hist": hist[: it.value + 1].copy(),
            "relres": relres.value}


def jacobi_pcg(labels, b, *, tol=1e-6, max_iter=10000):
    labels, lp, nx, ny, nz = _lab(labels)
    b, bp = _f64(b)
    x = np.zeros(labels.shape)
    it = ctypes.c_int(0)
    hist = np.zeros(max_iter + 1)
    relres = ctypes.c_double(0.0)
    st = lib().or_jacobi_pcg(lp, nx, ny, nz, bp, float(tol), int(max_iter), x.ctypes.data_as(_dp),
                             ctypes.byref(it), hist.ctypes.data_as(_dp), ctypes.byref(relres))
    return {"x": x, "iters": it.value, "status": st, "relres": relres.value,
            "res_hist": hist[: it.value + 1].copy()}


def network_transpose(labels, L, w, g):
    """P_net^T g: the input gradient of <g, P_net(I, r)> (the network is linear in r)."""
    _, gr = network_backward(labels, L, w, np.zeros(np.shape(labels)), g)
    return gr


def asymmetry(labels, L, w, x, y):
    """The relative asymmetry measure of the appendix's symmetry analysis:
    S(x, y; I) = |x . P(y) - y . P(x)| / sqrt(|x . P(x)| |y . P(y)|)."""
    px, py = network(labels, L, w, x), network(labels, L, w, y)
    xpy, ypx = float(np.sum(x * py)), float(np.sum(y * px))
    xpx, ypy = float(np.sum(x * px)), float(np.sum(y * py))
    return abs(xpy - ypx) / np.sqrt(abs(xpx) * abs(ypy))


def split_weights(w, L):
    """Views of the flat weight blob: dict level -> dict(block -> array)."""
    w = np.asarray(w, np.float64).ravel()
    out = {}
    per = 2 * CCONV_PARAMS + 2 * AFF_PARAMS
    for lvl in range(1, L):
        o = (lvl - 1) * per
        out[lvl] = {
            "cconv1": w[o:o + CCONV_PARAMS],
            "cconv2": w[o + CCONV_PARAMS:o + 2 * CCONV_PARAMS],
            "aff1": w[o + 2 * CCONV_PARAMS:o + 2 * CCONV_PARAMS + AFF_PARAMS],
            "aff2": w[o + 2 * CCONV_PARAMS + AFF_PARAMS:o + per],
        }
    o = (L - 1) * per
    out[L] = {"cconv1": w[o:o + CCONV_PARAMS]}
    return out
