"""Thin ctypes binding of libnpsolve.so (the C ABI of include/npsolve.h).

Argument marshalling only: device arrays are torch CUDA tensors passed by
``data_ptr()``, the stream is torch's current stream, host arrays are NumPy.
Every computation runs in the library's CUDA kernels; when the library cannot
be loaded every call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(HERE, "libnpsolve.so")

OK, BAD_ARG, BAD_DIMS, BAD_LABELS, NO_CONVERGENCE, BREAKDOWN, OOM, CUDA_ERROR = range(8)
FP32, BF16 = 0, 1
PATH_CACHED, PATH_CUDA_CORE, PATH_TENSOR = 0, 1, 2
RECURRENCE, EXPLICIT = 0, 1
NPSDO, PCG, FPCG = 0, 1, 2  # npsolve_config.method: Alg. 1, or (flexible) PCG with the network as preconditioner
STATUS_NAMES = ["OK", "BAD_ARG", "BAD_DIMS", "BAD_LABELS", "NO_CONVERGENCE", "BREAKDOWN", "OOM", "CUDA_ERROR"]


class NpsolveError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class _Config(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("n_ortho", ctypes.c_int), ("precision", ctypes.c_int),
                ("residual_mode", ctypes.c_int), ("kernel_path", ctypes.c_int), ("method", ctypes.c_int),
                ("symmetric", ctypes.c_int)]


_lib = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double

# Exported symbols and their argument types (mirrors include/npsolve.h).
SIGNATURES = {
    "npsolve_weight_count": ([_i], ctypes.c_size_t),
    "npsolve_create": ([ctypes.POINTER(_Config), _vp, ctypes.c_size_t, ctypes.POINTER(_vp)], _i),
    "npsolve_set_weights": ([_vp, _vp, ctypes.c_size_t], _i),
    "npsolve_get_weights": ([_vp, _vp, ctypes.c_size_t], _i),
    "npsolve_destroy": ([_vp], None),
    "npsolve_last_error": ([_vp], ctypes.c_char_p),
    "npsolve_solve": ([_vp, _vp, _i, _i, _i, _vp, _d, _i, _vp, _vp, ctypes.POINTER(_i), ctypes.POINTER(_d)], _i),
    "npsolve_solve_host": ([_vp, _vp, _i, _i, _i, _vp, _d, _i, _vp, _vp, ctypes.POINTER(_i), ctypes.POINTER(_d)],
                           _i),
    "npsolve_residual_history": ([_vp, _vp, _i, ctypes.POINTER(_i)], _i),
    "npsolve_apply_network": ([_vp, _vp, _i, _i, _i, _vp, _vp, _vp], _i),
    "npsolve_network_transpose": ([_vp, _vp, _i, _i, _i, _vp, _vp, _vp], _i),
    "npsolve_asymmetry": ([_vp, _vp, _i, _i, _i, _vp, _vp, _vp, ctypes.POINTER(_d), _vp], _i),
    "npsolve_network_intermediate": ([_vp, _vp, _i, _i, _i, _vp, _i, _i, _vp, _vp, _vp], _i),
    "npsolve_apply_laplacian": ([_vp, _i, _i, _i, _vp, _vp, _vp], _i),
    "npsolve_true_residual": ([_vp, _i, _i, _i, _vp, _vp, ctypes.POINTER(_d), _vp], _i),
    "npsolve_jacobi_pcg": ([_vp, _i, _i, _i, _vp, _d, _i, _vp, _vp, ctypes.POINTER(_i), ctypes.POINTER(_d)], _i),
    "npsolve_selftest_tensor_core": ([ctypes.POINTER(_d)], _i),
    "npsolve_network_vjp": ([_vp, _vp, _i, _i, _i, _vp, _vp, _vp, _vp, _vp], _i),
    "npsolve_loss_grad": ([_vp, _vp, _i, _i, _i, _vp, _vp, ctypes.POINTER(_d), _vp], _i),
    "npsolve_train_step": ([_vp, _i, _vp, _vp, _vp, ctypes.c_float, _vp, ctypes.POINTER(_d)], _i),
    "npsolve_lanczos_rhs": ([_vp, _i, _i, _i, _vp, _i, _i, _i, ctypes.c_ulonglong, _vp, _vp, _vp], _i),
    "npsolve_true_residual_noalloc": ([_vp, _i, _i, _i, _vp, _vp, ctypes.POINTER(_d), _vp], _i),
    "npsolve_workspace_bytes": ([_vp], ctypes.c_size_t),
    "npsolve_server_create": ([ctypes.POINTER(_Config), _vp, ctypes.c_size_t, ctypes.c_size_t, _i,
                               ctypes.POINTER(_vp)], _i),
    "npsolve_server_submit": ([_vp, _vp, _i, _i, _i, _vp, _vp, _d, _i, ctypes.POINTER(ctypes.c_longlong)], _i),
    "npsolve_server_poll": ([_vp, _vp, _i, ctypes.POINTER(_i)], _i),
    "npsolve_server_result": ([_vp, ctypes.c_longlong, ctypes.POINTER(_i), ctypes.POINTER(_d),
                               ctypes.POINTER(_i), ctypes.POINTER(_d), ctypes.POINTER(_d)], _i),
    "npsolve_server_stats": ([_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                              ctypes.POINTER(_i), ctypes.POINTER(_i)], _i),
    "npsolve_server_destroy": ([_vp], None),
    "npsolve_server_last_error": ([_vp], ctypes.c_char_p),
    "npsolve_profile_count": ([], _i),
    "npsolve_launch_count": ([_vp], ctypes.c_longlong),
    "npsolve_mixed_cells": ([_vp, _i], ctypes.c_longlong),
    "npsolve_level1_work": ([_vp, _i, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)], _i),
    "npsolve_profile_name": ([_i], ctypes.c_char_p),
    "npsolve_set_profiling": ([_vp, _i], _i),
    "npsolve_get_profile": ([_vp, _vp, _vp], _i),
}


def lib_path() -> str:
    return _LIB_PATH


def load_library():
    """Load libnpsolve.so (raises OSError when it is missing or unloadable)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise OSError(f"{_LIB_PATH} not built; run paper_2310_00177_b300/build.py")
        lib = ctypes.CDLL(_LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype=None, name="tensor"):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA torch tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _dims(labels):
    if labels.dim() != 3:
        raise ValueError("labels must be (nz, ny, nx)")
    nz, ny, nx = labels.shape
    return int(nx), int(ny), int(nz)


def _check(st, h=None):
    if st != OK:
        msg = load_library().npsolve_last_error(h).decode()
        raise NpsolveError(st, msg)


def weight_count(levels: int) -> int:
    return int(load_library().npsolve_weight_count(levels))


class Solver:
    """A solver handle: network weights + device workspace (npsolve_t)."""

    def __init__(self, weights, levels=4, n_ortho=2, precision=FP32, residual_mode=RECURRENCE,
                 kernel_path=PATH_CACHED, method=NPSDO, symmetric=False):
        lib = load_library()
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32).ravel())
        cfg = _Config(levels, n_ortho, precision, residual_mode, kernel_path, method, int(bool(symmetric)))
        h = ctypes.c_void_p()
        st = lib.npsolve_create(ctypes.byref(cfg), w.ctypes.data_as(_vp), w.size, ctypes.byref(h))
        if st != OK:
            raise NpsolveError(st, lib.npsolve_last_error(None).decode())
        self._h = h
        self.levels, self.n_ortho, self.precision, self.residual_mode = levels, n_ortho, precision, residual_mode
        self.kernel_path, self.method, self.symmetric = kernel_path, method, bool(symmetric)

    def close(self):
        if getattr(self, "_h", None):
            load_library().npsolve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_weights(self, weights):
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32).ravel())
        _check(load_library().npsolve_set_weights(self._h, w.ctypes.data_as(_vp), w.size), self._h)

    def get_weights(self):
        n = weight_count(self.levels)
        w = np.empty(n, np.float32)
        _check(load_library().npsolve_get_weights(self._h, w.ctypes.data_as(_vp), n), self._h)
        return w

    def solve(self, labels, b, tol=1e-6, max_iter=1000, x=None):
        """NPSDO solve on device tensors.  Returns (x, iters, rel_residual, status);
        status is OK, NO_CONVERGENCE or BREAKDOWN, other failures raise."""
        import torch

        nx, ny, nz = _dims(labels)
        if x is None:
            x = torch.empty(labels.shape, dtype=torch.float64, device=labels.device)
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = load_library().npsolve_solve(self._h, _ptr(labels, torch.uint8, "labels"), nx, ny, nz,
                                          _ptr(b, torch.float32, "b"), float(tol), int(max_iter), _stream(),
                                          _ptr(x, torch.float64, "x"), ctypes.byref(it), ctypes.byref(rr))
        if st not in (OK, NO_CONVERGENCE, BREAKDOWN):
            _check(st, self._h)
        return x, it.value, rr.value, st

    def solve_host(self, labels, b, tol=1e-6, max_iter=1000, x=None):
        """The same solve on host NumPy arrays (copies inside the library call)."""
        labels = np.ascontiguousarray(labels, dtype=np.uint8)
        b = np.ascontiguousarray(b, dtype=np.float32)
        nz, ny, nx = labels.shape
        if x is None:
            x = np.empty(labels.shape, np.float64)
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = load_library().npsolve_solve_host(self._h, labels.ctypes.data_as(_vp), nx, ny, nz,
                                               b.ctypes.data_as(_vp), float(tol), int(max_iter), _stream(),
                                               x.ctypes.data_as(_vp), ctypes.byref(it), ctypes.byref(rr))
        if st not in (OK, NO_CONVERGENCE, BREAKDOWN):
            _check(st, self._h)
        return x, it.value, rr.value, st

    def mixed_cells(self, level):
        """Cells of `level` with a non-uniform image window in the last setup (-1 if unknown)."""
        return int(load_library().npsolve_mixed_cells(self._h, level))

    def level1_work(self, which):
        """(cells, mixed cells) of the units the level-1 CConv1 (which=0) or
        CConv2 (which=1) processed in the last solve (occupancy-aware sparsity)."""
        c, m = ctypes.c_longlong(0), ctypes.c_longlong(0)
        _check(load_library().npsolve_level1_work(self._h, int(which), ctypes.byref(c), ctypes.byref(m)), self._h)
        return c.value, m.value

    def launch_count(self):
        """Kernels enqueued by this handle since creation."""
        return int(load_library().npsolve_launch_count(self._h))

    def network_vjp(self, labels, r, gz, want_grad_r=True):
        """Backward of z = P_net(I, r) for the cotangent gz: (grad_w numpy, grad_r tensor or None)."""
        import torch

        nx, ny, nz = _dims(labels)
        gw = np.zeros(weight_count(self.levels), np.float32)
        gr = torch.empty(labels.shape, dtype=torch.float32, device=labels.device) if want_grad_r else None
        _check(load_library().npsolve_network_vjp(
            self._h, _ptr(labels, torch.uint8, "labels"), nx, ny, nz, _ptr(r, torch.float32, "r"),
            _ptr(gz, torch.float32, "gz"), gw.ctypes.data_as(_vp),
            _ptr(gr, torch.float32, "grad_r") if gr is not None else None, _stream()), self._h)
        return gw, gr

    def loss_grad(self, labels, b, want_grad=True):
        """Loss ||b - A P_net(I, b)|| and its weight gradient (numpy) of one system."""
        import torch

        nx, ny, nz = _dims(labels)
        loss = ctypes.c_double(0.0)
        gw = np.zeros(weight_count(self.levels), np.float32) if want_grad else None
        _check(load_library().npsolve_loss_grad(
            self._h, _ptr(labels, torch.uint8, "labels"), nx, ny, nz, _ptr(b, torch.float32, "b"), _stream(),
            ctypes.byref(loss), gw.ctypes.data_as(_vp) if gw is not None else None), self._h)
        return loss.value, gw

    def train_step(self, labels_list, b_list, lr=1e-3):
        """One Adam step on a batch of systems (lists of device tensors); returns the mean loss."""
        import torch

        n = len(labels_list)
        labs = (ctypes.c_void_p * n)(*[_ptr(l, torch.uint8, "labels").value for l in labels_list])
        bs = (ctypes.c_void_p * n)(*[_ptr(x, torch.float32, "b").value for x in b_list])
        dims = np.ascontiguousarray(np.array([_dims(l) for l in labels_list], np.int32).ravel())
        loss = ctypes.c_double(0.0)
        _check(load_library().npsolve_train_step(self._h, n, labs, dims.ctypes.data_as(_vp), bs, float(lr),
                                                 _stream(), ctypes.byref(loss)), self._h)
        return loss.value

    def set_profiling(self, on=True):
        _check(load_library().npsolve_set_profiling(self._h, int(bool(on))), self._h)

    def profile(self):
        """Per kernel class: (total device ms, timed launches) of the profiled solves."""
        lib = load_library()
        n = lib.npsolve_profile_count()
        ms = np.zeros(n, np.float64)
        cnt = np.zeros(n, np.int64)
        _check(lib.npsolve_get_profile(self._h, ms.ctypes.data_as(_vp), cnt.ctypes.data_as(_vp)), self._h)
        return {lib.npsolve_profile_name(i).decode(): (float(ms[i]), int(cnt[i])) for i in range(n)}

    def residual_history(self, cap=100000):
        out = np.zeros(cap, np.float64)
        cnt = ctypes.c_int(0)
        _check(load_library().npsolve_residual_history(self._h, out.ctypes.data_as(_vp), cap, ctypes.byref(cnt)),
               self._h)
        return out[: cnt.value].copy()

    def apply_network(self, labels, r, z=None):
        import torch

        nx, ny, nz = _dims(labels)
        if z is None:
            z = torch.empty(labels.shape, dtype=torch.float32, device=labels.device)
        _check(load_library().npsolve_apply_network(self._h, _ptr(labels, torch.uint8, "labels"), nx, ny, nz,
                                                    _ptr(r, torch.float32, "r"), _ptr(z, torch.float32, "z"),
                                                    _stream()), self._h)
        return z

    def network_transpose(self, labels, g, out=None):
        """P_net^T g (the adjoint of apply_network)."""
        import torch

        nx, ny, nz = _dims(labels)
        if out is None:
            out = torch.empty(labels.shape, dtype=torch.float32, device=labels.device)
        _check(load_library().npsolve_network_transpose(self._h, _ptr(labels, torch.uint8, "labels"), nx, ny, nz,
                                                        _ptr(g, torch.float32, "g"), _ptr(out, torch.float32, "out"),
                                                        _stream()), self._h)
        return out

    def asymmetry(self, labels, x, y):
        """The relative asymmetry measure S(x, y; I) of the network and its four
        dots (x.P(y), x.P(x), y.P(x), y.P(y))."""
        import torch

        nx, ny, nz = _dims(labels)
        S = ctypes.c_double(0.0)
        dots = np.zeros(4, np.float64)
        _check(load_library().npsolve_asymmetry(self._h, _ptr(labels, torch.uint8, "labels"), nx, ny, nz,
                                                _ptr(x, torch.float32, "x"), _ptr(y, torch.float32, "y"), _stream(),
                                                ctypes.byref(S), dots.ctypes.data_as(_vp)), self._h)
        return S.value, dots

    def network_intermediate(self, labels, r, level, which):
        """which: 'x1', 'r2', 'x2', 'x', 'r1'.  Returns (field, (c1, c2))."""
        import torch

        code = {"x1": 0, "r2": 1, "x2": 2, "x": 3, "r1": 4}[which]
        nx, ny, nz = _dims(labels)
        s = 1 << (level - 1)
        out = torch.empty((nz // s, ny // s, nx // s), dtype=torch.float32, device=labels.device)
        c12 = np.zeros(2, np.float64)
        _check(load_library().npsolve_network_intermediate(
            self._h, _ptr(labels, torch.uint8, "labels"), nx, ny, nz, _ptr(r, torch.float32, "r"), level, code,
            _ptr(out, torch.float32, "out"), c12.ctypes.data_as(_vp), _stream()), self._h)
        return out, (float(c12[0]), float(c12[1]))


def apply_laplacian(labels, d, q=None):
    import torch

    nx, ny, nz = _dims(labels)
    if q is None:
        q = torch.empty(labels.shape, dtype=torch.float32, device=labels.device)
    _check(load_library().npsolve_apply_laplacian(_ptr(labels, torch.uint8, "labels"), nx, ny, nz,
                                                  _ptr(d, torch.float32, "d"), _ptr(q, torch.float32, "q"),
                                                  _stream()))
    return q


def true_residual(labels, b, x):
    import torch

    nx, ny, nz = _dims(labels)
    rr = ctypes.c_double(0.0)
    _check(load_library().npsolve_true_residual(_ptr(labels, torch.uint8, "labels"), nx, ny, nz,
                                                _ptr(b, torch.float32, "b"), _ptr(x, torch.float64, "x"),
                                                ctypes.byref(rr), _stream()))
    return rr.value


def jacobi_pcg(labels, b, tol=1e-6, max_iter=100000, x=None):
    import torch

    nx, ny, nz = _dims(labels)
    if x is None:
        x = torch.empty(labels.shape, dtype=torch.float64, device=labels.device)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = load_library().npsolve_jacobi_pcg(_ptr(labels, torch.uint8, "labels"), nx, ny, nz,
                                           _ptr(b, torch.float32, "b"), float(tol), int(max_iter), _stream(),
                                           _ptr(x, torch.float64, "x"), ctypes.byref(it), ctypes.byref(rr))
    if st not in (OK, NO_CONVERGENCE, BREAKDOWN):
        _check(st)
    return x, it.value, rr.value, st


def selftest_tensor_core():
    """Max abs error of one tcgen05 BF16 MMA (A in TMEM, B in smem) vs CUDA cores."""
    e = ctypes.c_double(-1.0)
    _check(load_library().npsolve_selftest_tensor_core(ctypes.byref(e)))
    return e.value


class NetworkFunction:
    """torch.autograd.Function of z = P_net(I, r) with respect to the weights
    and r, whose backward is the library's hand-written kernel
    (npsolve_network_vjp).  Usage: NetworkFunction.apply(weights, labels, r, solver)."""

    _fn = None

    @staticmethod
    def get():
        if NetworkFunction._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, weights, labels, r, solver):
                    solver.set_weights(weights.detach().cpu().numpy())
                    ctx.save_for_backward(labels, r)
                    ctx.solver = solver
                    return solver.apply_network(labels, r.detach().contiguous().float())

                @staticmethod
                def backward(ctx, gz):
                    labels, r = ctx.saved_tensors
                    gw, gr = ctx.solver.network_vjp(labels, r.detach().contiguous().float(),
                                                    gz.detach().contiguous().float())
                    return torch.from_numpy(gw), None, gr, None

            NetworkFunction._fn = _F
        return NetworkFunction._fn

    @staticmethod
    def apply(weights, labels, r, solver):
        return NetworkFunction.get().apply(weights, labels, r, solver)


def lanczos_rhs(labels, start, m=48, k=32, count=4, seed=0):
    """Random normalised combinations of the k lowest Ritz vectors of A from m
    Lanczos steps (device tensors); returns (rhs [count, *shape], ritz values)."""
    import torch

    nx, ny, nz = _dims(labels)
    out = torch.empty((count,) + tuple(labels.shape), dtype=torch.float32, device=labels.device)
    vals = np.zeros(k, np.float64)
    _check(load_library().npsolve_lanczos_rhs(_ptr(labels, torch.uint8, "labels"), nx, ny, nz,
                                              _ptr(start, torch.float32, "start"), int(m), int(k), int(count),
                                              int(seed), _ptr(out, torch.float32, "out"),
                                              vals.ctypes.data_as(_vp), _stream()))
    return out, vals


class Server:
    """Continuous-batching solve server (npsolve_server_*): submit host arrays,
    poll for finished ids, fetch results."""

    def __init__(self, weights, levels=4, n_ortho=2, precision=BF16, residual_mode=RECURRENCE,
                 kernel_path=PATH_CACHED, hbm_budget_bytes=150 << 30, max_active=16, method=NPSDO,
                 symmetric=False):
        lib = load_library()
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32).ravel())
        cfg = _Config(levels, n_ortho, precision, residual_mode, kernel_path, method, int(bool(symmetric)))
        h = ctypes.c_void_p()
        st = lib.npsolve_server_create(ctypes.byref(cfg), w.ctypes.data_as(_vp), w.size, int(hbm_budget_bytes),
                                       int(max_active), ctypes.byref(h))
        if st != OK:
            raise NpsolveError(st, lib.npsolve_last_error(None).decode())
        self._h = h
        self.levels = levels
        self._alive = {}

    def _check(self, st):
        if st != OK:
            raise NpsolveError(st, load_library().npsolve_server_last_error(self._h).decode())

    def submit(self, labels, b, x=None, tol=1e-6, max_iter=1000):
        """Queue a solve; labels (uint8), b (float32) and x (float64 output, or
        None) are host arrays kept alive by the server object until the result
        is read (pinned arrays give the fastest copies)."""
        labels = np.ascontiguousarray(labels, dtype=np.uint8)
        b = np.ascontiguousarray(b, dtype=np.float32)
        if x is not None:
            assert x.dtype == np.float64 and x.flags["C_CONTIGUOUS"] and x.shape == labels.shape
        nz, ny, nx = labels.shape
        rid = ctypes.c_longlong(-1)
        self._check(load_library().npsolve_server_submit(
            self._h, labels.ctypes.data_as(_vp), nx, ny, nz, b.ctypes.data_as(_vp),
            x.ctypes.data_as(_vp) if x is not None else None, float(tol), int(max_iter), ctypes.byref(rid)))
        self._alive[rid.value] = (labels, b, x)
        return rid.value

    def poll(self, cap=1024):
        ids = np.zeros(cap, np.int64)
        cnt = ctypes.c_int(0)
        self._check(load_library().npsolve_server_poll(self._h, ids.ctypes.data_as(_vp), cap, ctypes.byref(cnt)))
        return [int(v) for v in ids[:cnt.value]]

    def result(self, rid):
        """(x or None, iters, rel_residual, status, queue_ms, service_ms)."""
        it, st = ctypes.c_int(0), ctypes.c_int(0)
        rr, qm, sm = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
        self._check(load_library().npsolve_server_result(self._h, int(rid), ctypes.byref(it), ctypes.byref(rr),
                                                         ctypes.byref(st), ctypes.byref(qm), ctypes.byref(sm)))
        _, _, x = self._alive.pop(int(rid), (None, None, None))
        return x, it.value, rr.value, st.value, qm.value, sm.value

    def stats(self):
        r, p = ctypes.c_size_t(0), ctypes.c_size_t(0)
        a, q = ctypes.c_int(0), ctypes.c_int(0)
        self._check(load_library().npsolve_server_stats(self._h, ctypes.byref(r), ctypes.byref(p), ctypes.byref(a),
                                                        ctypes.byref(q)))
        return {"reserved": r.value, "peak_reserved": p.value, "active": a.value, "queued": q.value}

    def close(self):
        if getattr(self, "_h", None):
            load_library().npsolve_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
