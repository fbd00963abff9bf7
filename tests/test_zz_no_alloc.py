"""The allocation-free true-residual entry point, called through the C ABI.

npsolve_true_residual_noalloc serves callers that must not allocate device
memory when they check a solution (a simulation frame loop with all GPU
memory reserved up front, a plug-in whose host owns the device memory).  It
must give the same FP64 relative residual as npsolve_true_residual, call
after call (its scratch array is shared and reused), and reject grids larger
than its 16,777,216-cell maximum.  The two entry points reduce in different
orders (different block counts), so they agree to FP64 rounding, 1e-12
relative."""
import ctypes

import numpy as np
import pytest

from paper_2310_00177_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _lib():
    from paper_2310_00177_b300 import binding

    return binding.load_library()


def _call(fn, lab, b, x):
    nz, ny, nx = lab.shape
    out = ctypes.c_double(-1.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = fn(ctypes.c_void_p(lab.data_ptr()), nx, ny, nz, ctypes.c_void_p(b.data_ptr()),
            ctypes.c_void_p(x.data_ptr()), ctypes.byref(out), stream)
    return st, out.value


def test_no_alloc_true_residual_matches_the_allocating_entry_point():
    lib = _lib()
    for k, (n, seed) in enumerate([(64, 11), (96, 12)]):  # two calls in a row, different problems
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


def test_no_alloc_true_residual_rejects_grids_above_its_maximum():
    lib = _lib()
    shape = (256, 256, 512)  # 33,554,432 cells > 16,777,216
    lab = torch.zeros(shape, dtype=torch.uint8, device="cuda")
    b = torch.zeros(shape, dtype=torch.float32, device="cuda")
    x = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st, _ = _call(lib.npsolve_true_residual_noalloc, lab, b, x)
    assert st == 2  # NPSOLVE_BAD_DIMS
    assert b"maximum" in lib.npsolve_last_error(None)
