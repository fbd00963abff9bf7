"""B300-native neural-preconditioned Poisson solver (NPSDO, arXiv 2310.00177).

The compute path is the CUDA library ``libnpsolve.so`` (hand-written kernels
for sm_103a behind a C ABI, declared in ``include/npsolve.h``); this package is
a thin ctypes binding to it.  The binding is imported lazily so that the
input generators in ``synth`` can be used without a GPU.
"""


def __getattr__(name):
    if name in ("Solver", "NpsolveError", "load_library", "lib_path"):
        from . import binding

        return getattr(binding, name)
    raise AttributeError(name)
