"""ctypes loader for the in-tree C-ABI library (``include/pipe_poisson.h``).

Argument marshalling only: every entry point is a direct call into
``libpipepoisson.so``.  If the library is missing this raises; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int64, c_size_t, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libpipepoisson.so")

PIPE_OK = 0
PIPE_EINVAL = 1
PIPE_ENOMEM = 2
PIPE_EUNSUPPORTED = 3
PIPE_ECUDA = 4
PIPE_ETIMEOUT = 5
PIPE_ENODEVICE = 6
PIPE_F32 = 0
PIPE_F64 = 1
PIPE_F32_C16 = 2          # FP32 arithmetic, complex-FP16 spectra with per-slab scales


class PipeGeometry(ctypes.Structure):
    _fields_ = [("a", c_double), ("b", c_double), ("x0", c_double), ("y0", c_double),
                ("modes_m", c_int), ("modes_n", c_int)]


class PipeGrid(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int),
                ("hx", c_double), ("hy", c_double), ("hz", c_double), ("dtype", c_int)]


H = c_void_p  # pipe_handle*

SIGNATURES = {
    "pipe_green_setup": (c_int, [POINTER(PipeGeometry), POINTER(PipeGrid), c_int, POINTER(H)]),
    "pipe_free_space_setup": (c_int, [POINTER(PipeGrid), c_double, POINTER(H)]),
    "pipe_banded_setup": (c_int, [POINTER(PipeGeometry), POINTER(PipeGrid), c_int, c_int, POINTER(H)]),
    "pipe_poisson_solve": (c_int, [H, c_void_p, c_void_p, c_void_p]),
    "pipe_poisson_adjoint": (c_int, [H, c_void_p, c_void_p, c_void_p]),
    "pipe_poisson_solve_host": (c_int, [H, c_void_p, c_void_p, c_void_p]),
    "pipe_poisson_solve_noalloc": (c_int, [H, c_void_p, c_void_p, c_void_p]),
    "pipe_poisson_solve_host_stream": (c_int, [H, POINTER(c_void_p), POINTER(c_void_p), c_int, c_void_p]),
    "pipe_poisson_solve_batched": (c_int, [POINTER(H), POINTER(c_void_p), POINTER(c_void_p), c_int,
                                           c_void_p]),
    "pipe_electric_field": (c_int, [H, c_void_p, c_void_p, c_void_p]),
    "pipe_batch_status": (c_int, [POINTER(H), c_int]),
    "pipe_batch_inject_fault": (c_int, [POINTER(H), c_int, c_int, ctypes.c_longlong]),
    "pipe_batch_plan_info": (c_int, [POINTER(H), c_int, POINTER(c_int), POINTER(c_int)]),
    "pipe_batch_side_streams": (c_int, [POINTER(H), c_int, POINTER(c_int)]),
    "pipe_batch_select_streams": (c_int, [POINTER(H), c_int, c_int]),
    "pipe_batch_grouped": (c_int, [POINTER(H), c_int, POINTER(c_int), POINTER(c_int)]),
    "pipe_batch_select_groups": (c_int, [POINTER(H), c_int, c_int]),
    "pipe_batch_select": (c_int, [POINTER(H), c_int, c_int, c_int]),
    "pipe_green_spectrum": (c_int, [H, POINTER(c_double), c_size_t]),
    "pipe_stage_z_forward": (c_int, [H, c_void_p, c_void_p, c_int, c_void_p]),
    "pipe_stage_transverse": (c_int, [H, c_void_p, c_int, c_void_p]),
    "pipe_stage_z_inverse": (c_int, [H, c_void_p, c_void_p, c_int, c_void_p]),
    "pipe_stage_modes": (c_int, [H, c_int, c_void_p, c_void_p, c_void_p]),
    "pipe_mode_layout": (c_int, [H, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int),
                                 POINTER(c_int)]),
    "pipe_mode_spectrum": (c_int, [H, POINTER(c_double), c_size_t]),
    "pipe_autotune": (c_int, [H, c_void_p]),
    "pipe_get_plan": (c_int, [H, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int),
                              POINTER(c_int)]),
    "pipe_set_plan": (c_int, [H, c_int, c_int, c_int, c_int, c_int]),
    "pipe_status": (c_int, [H]),
    "pipe_inject_stage_fault": (c_int, [H, c_int, ctypes.c_longlong]),
    "pipe_cic_deposit": (c_int, [H, c_void_p, c_int64, c_double, c_void_p, c_void_p]),
    "pipe_cic_gather_grad": (c_int, [H, c_void_p, c_int64, c_double, c_void_p, c_void_p, c_void_p]),
    "pipe_green_destroy": (None, [H]),
    "pipe_strerror": (c_char_p, [c_int]),
    "pipe_selftest_twiddles": (c_double, []),
    "pipe_version": (c_char_p, []),
}

_LIB = None


class PipeError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _LIB.pipe_strerror(status).decode() if _LIB is not None else str(status)
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


def load(path: str | None = None):
    """Load (once) and return the library with typed entry points."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or LIBPATH
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with `python -m paper_1111_4971_gb300.build` "
            "(or __graft_entry__.build()); there is no fallback implementation")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def check(status: int, where: str):
    if status != PIPE_OK:
        raise PipeError(status, where)
