"""The allocation-free true-residual entry point, called through the C ABI.

npsolve_true_residual_noalloc serves callers that must not allocate device
memory when they check a solution (a simulation frame loop with all GPU
memory reserved up front, a plug-in whose host owns the device memory).  It
must give the same FP64 relative residual as npsolve_true_residual, call
after call (its scratch array is shared and reused), leave the device's
memory untouched, and reject grids larger than its 16,777,216-cell maximum.

Both entry points do the same FP64 operations per fluid cell; only the order
of the cross-block reduction differs (different block counts).  Each squared
sum then carries a relative rounding error of at most about (number of
partial sums) * 2^-53 ~ 1e-12, at random x (residual of order 1) and at a
converged solve's x (relative residual ~1e-6) alike, since the per-cell
residuals are formed identically before the reduction.  Tolerance: 1e-12
relative on the square root of their ratio.

This file is collected last, so a run that stops at its first failure has
run every other test already; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2310_00177_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _binding():
    from paper_2310_00177_b300 import binding

    return binding


def _call(fn, lab, b, x):
    nz, ny, nx = lab.shape
    out = ctypes.c_double(-1.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = fn(ctypes.c_void_p(lab.data_ptr()), nx, ny, nz, ctypes.c_void_p(b.data_ptr()),
            ctypes.c_void_p(x.data_ptr()), ctypes.byref(out), stream)
    return st, out.value


def _memory_state():
    """Free device memory (cudaMemGetInfo) and the default memory pool's
    reserved and used bytes (the pool cudaMallocAsync draws from)."""
    from cuda.bindings import runtime as rt

    dev = torch.cuda.current_device()
    err, pool = rt.cudaDeviceGetDefaultMemPool(dev)
    assert err == rt.cudaError_t.cudaSuccess
    vals = []
    for attr in (rt.cudaMemPoolAttr.cudaMemPoolAttrReservedMemCurrent, rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemCurrent):
        err, v = rt.cudaMemPoolGetAttribute(pool, attr)
        assert err == rt.cudaError_t.cudaSuccess
        vals.append(int(v))
    torch.cuda.synchronize()
    return (torch.cuda.mem_get_info()[0], *vals)


def test_no_alloc_true_residual_matches_the_allocating_entry_point():
    lib = _binding().load_library()
    for n, seed in [(64, 11), (96, 12)]:  # two calls in a row, different problems
        lab_np = synth.slosh_scene(n, seed)
        rng = np.random.default_rng(seed)
        lab = torch.from_numpy(lab_np).cuda()
        b = torch.from_numpy(synth.rhs_normal(lab_np, seed + 1).astype(np.float32)).cuda()
        x = torch.from_numpy(rng.standard_normal(lab_np.shape) * 0.1).cuda()
        st_ref, ref = _call(lib.npsolve_true_residual, lab, b, x)
        st_na, val = _call(lib.npsolve_true_residual_noalloc, lab, b, x)
        assert st_ref == 0 and st_na == 0
        assert val == pytest.approx(ref, rel=1e-12)
        assert val > 0.0


def test_no_alloc_true_residual_at_a_converged_solution():
    # the case callers have: x from a solve stopped at 1e-6, where b - A x is
    # small compared with b and A x
    b_ = _binding()
    lib = b_.load_library()
    lab_np = synth.slosh_scene(64, 2000)
    rhs_np = synth.rhs_normal(lab_np, 2001).astype(np.float32)
    lab, b = torch.from_numpy(lab_np).cuda(), torch.from_numpy(rhs_np).cuda()
    s = b_.Solver(synth.init_weights(4, 7).astype(np.float32), levels=4, n_ortho=2)
    x, _, relres, st = s.solve(lab, b, 1e-6, 1000)
    s.close()
    assert st == b_.OK and 0 < relres < 1e-6
    st_ref, ref = _call(lib.npsolve_true_residual, lab, b, x)
    st_na, val = _call(lib.npsolve_true_residual_noalloc, lab, b, x)
    assert st_ref == 0 and st_na == 0
    assert 0 < val < 1e-6
    assert val == pytest.approx(ref, rel=1e-12)


def test_no_alloc_true_residual_allocates_nothing_and_repeats_bitwise():
    lib = _binding().load_library()
    lab_np = synth.slosh_scene(96, 21)
    lab = torch.from_numpy(lab_np).cuda()
    b = torch.from_numpy(synth.rhs_normal(lab_np, 22).astype(np.float32)).cuda()
    x = torch.from_numpy(np.random.default_rng(23).standard_normal(lab_np.shape) * 0.1).cuda()
    st, first = _call(lib.npsolve_true_residual_noalloc, lab, b, x)  # looks the array up on this device
    assert st == 0
    before = _memory_state()
    vals = []
    for _ in range(3):
        st, v = _call(lib.npsolve_true_residual_noalloc, lab, b, x)
        assert st == 0
        vals.append(v)
    after = _memory_state()
    assert after == before  # no device memory taken, from the pool or outside it
    assert all(v == first for v in vals)  # the shared array's reuse changes nothing


def test_no_alloc_true_residual_rejects_grids_above_its_maximum():
    lib = _binding().load_library()
    shape = (256, 256, 512)  # 33,554,432 cells > 16,777,216
    lab = torch.zeros(shape, dtype=torch.uint8, device="cuda")
    b = torch.zeros(shape, dtype=torch.float32, device="cuda")
    x = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st, _ = _call(lib.npsolve_true_residual_noalloc, lab, b, x)
    assert st == 2  # NPSOLVE_BAD_DIMS
    assert b"maximum" in lib.npsolve_last_error(None)
