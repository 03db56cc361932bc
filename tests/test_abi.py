"""The C-ABI library loads and exports what include/pipe_poisson.h declares.

CPU only: no call here launches a kernel (argument validation runs before any
CUDA call).
"""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1111_4971_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pipe_poisson.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pipe_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def L():
    from paper_1111_4971_gb300 import build
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported_and_bound(L):
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIBPATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (pipe_[a-z0-9_]+)", out))
    for n in names:
        assert n in exported, n
        assert n in _lib.SIGNATURES, n
        assert getattr(L, n) is not None


def test_compile_time_twiddles(L):
    assert L.pipe_selftest_twiddles() <= 4.5e-16  # two ulp at 1.0


def test_strerror_and_version(L):
    assert L.pipe_strerror(0) == b"ok"
    assert b"unsupported" in L.pipe_strerror(3)
    assert b"sm_103a" in L.pipe_version()


def _setup(L, geo, grid, igf=1):
    h = ctypes.c_void_p()
    st = L.pipe_green_setup(ctypes.byref(geo) if geo is not None else None,
                            ctypes.byref(grid) if grid is not None else None, igf, ctypes.byref(h))
    return st, h


def test_setup_validation_without_gpu(L):
    G, P = _lib.PipeGeometry, _lib.PipeGrid
    good_geo = G(1.0, 1.0, 1 / 256, 1 / 256, 20, 20)
    good = P(128, 128, 256, 1 / 128, 1 / 128, 0.1, 0)
    cases = [
        (None, good, 1, _lib.PIPE_EINVAL),
        (good_geo, None, 1, _lib.PIPE_EINVAL),
        (good_geo, good, 7, _lib.PIPE_EINVAL),                           # bad igf
        (G(-1.0, 1.0, 0, 0, 20, 20), good, 1, _lib.PIPE_EINVAL),         # a <= 0
        (good_geo, P(128, 128, 256, 0.0, 1 / 128, 0.1, 0), 1, _lib.PIPE_EINVAL),   # h = 0
        (good_geo, P(128, 128, 256, 1 / 128, 1 / 128, 0.1, 5), 1, _lib.PIPE_EINVAL),  # dtype
        (G(1.0, 1.0, 0.5, 0.0, 20, 20), good, 1, _lib.PIPE_EINVAL),      # mesh leaves the pipe
        (G(1.0, 1.0, 0.0, 0.0, 0, 20), good, 1, _lib.PIPE_EINVAL),       # no modes
        # sizes neither form takes: not a power of two nor a multiple of 16
        (good_geo, P(100, 100, 256, 1 / 100, 1 / 100, 0.1, 0), 1, _lib.PIPE_EUNSUPPORTED),
        (good_geo, P(128, 72, 256, 1 / 128, 1 / 72, 0.1, 0), 1, _lib.PIPE_EUNSUPPORTED),   # nx != ny, 72
        (good_geo, P(128, 128, 4096, 1 / 128, 1 / 128, 0.1, 0), 1, _lib.PIPE_EUNSUPPORTED),
        # complex-FP16 spectra: transform form only, powers of two
        (good_geo, P(96, 96, 256, 1 / 96, 1 / 96, 0.1, 2), 1, _lib.PIPE_EUNSUPPORTED),
        # a window wider than 64 with more modes than the mode form holds
        (G(2.0, 2.0, 0.5, 0.5, 40, 40), P(128, 128, 32, 0.01, 0.01, 0.1, 0), 1,
         _lib.PIPE_EUNSUPPORTED),
        # 2x0/h not an integer (a window for the transform form), 33 modes
        (G(1.0, 1.0, 0.3 / 128, 0.5 / 128, 33, 20), good, 1, _lib.PIPE_EUNSUPPORTED),
    ]
    for geo, grid, igf, want in cases:
        st, h = _setup(L, geo, grid, igf)
        assert st == want, (geo, grid, igf, st)
        assert not h.value


def test_null_handle_and_pointers(L):
    assert L.pipe_poisson_solve(None, None, None, None) == _lib.PIPE_EINVAL
    assert L.pipe_poisson_adjoint(None, None, None, None) == _lib.PIPE_EINVAL
    assert L.pipe_poisson_solve_host(None, None, None, None) == _lib.PIPE_EINVAL
    assert L.pipe_green_spectrum(None, None, 0) == _lib.PIPE_EINVAL
    assert L.pipe_mode_spectrum(None, None, 0) == _lib.PIPE_EINVAL
    assert L.pipe_stage_modes(None, 0, None, None, None) == _lib.PIPE_EINVAL
    v = [ctypes.c_int() for _ in range(5)]
    assert L.pipe_mode_layout(None, *[ctypes.byref(x) for x in v]) == _lib.PIPE_EINVAL
    L.pipe_green_destroy(None)


def test_status_fault_hook_and_batch_stream_entry_points_refuse_bad_arguments(L):
    """Argument checks that come before any CUDA call (no device needed)."""
    import ctypes
    assert L.pipe_status(None) == _lib.PIPE_EINVAL
    assert L.pipe_inject_stage_fault(None, 0, 100) == _lib.PIPE_EINVAL
    n = ctypes.c_int(-1)
    assert L.pipe_batch_side_streams(None, 1, ctypes.byref(n)) == _lib.PIPE_EINVAL
    assert n.value == -1
    assert L.pipe_batch_select_streams(None, 1, 2) == _lib.PIPE_EINVAL
    hs = (ctypes.c_void_p * 1)(None)
    assert L.pipe_batch_side_streams(hs, 1, None) == _lib.PIPE_EINVAL
    assert L.pipe_batch_select_streams(hs, 1, 2) == _lib.PIPE_EINVAL       # null handle
    assert L.pipe_batch_select_streams(hs, 0, 2) == _lib.PIPE_EINVAL       # empty set
    assert L.pipe_batch_grouped(None, 1, ctypes.byref(n), None) == _lib.PIPE_EINVAL
    assert L.pipe_batch_grouped(hs, 1, None, None) == _lib.PIPE_EINVAL
    assert L.pipe_batch_select_groups(hs, 1, 1) == _lib.PIPE_EINVAL        # null handle
    assert L.pipe_batch_select_groups(None, 1, 2) == _lib.PIPE_EINVAL


def test_banded_setup_validation_without_gpu(L):
    G, P = _lib.PipeGeometry, _lib.PipeGrid
    cc = G(1.0, 1.0, 0.5 / 128, 0.5 / 128, 20, 20)
    good = P(128, 128, 256, 1 / 128, 1 / 128, 0.1, 0)
    cases = [
        (cc, good, -1, _lib.PIPE_EINVAL),                                  # negative band
        (cc, good, 256, _lib.PIPE_EINVAL),                                 # band >= nz
        # meshes neither banded form takes: more than 32 modes (beyond the
        # mode-space form) with x0 = 0 (s = 0) or an FP64 128^2 plane (beyond
        # the banded transform kernels)
        (G(1.0, 1.0, 0.0, 0.0, 40, 40), good, 1, _lib.PIPE_EUNSUPPORTED),
        (G(1.0, 1.0, 0.5 / 128, 0.5 / 128, 40, 40), P(128, 128, 256, 1 / 128, 1 / 128, 0.1, 1), 1,
         _lib.PIPE_EUNSUPPORTED),
    ]
    for geo, grid, n_nb, want in cases:
        h = ctypes.c_void_p()
        st = L.pipe_banded_setup(ctypes.byref(geo), ctypes.byref(grid), 1, n_nb, ctypes.byref(h))
        assert st == want, (n_nb, st)
        assert not h.value


def test_missing_library_fails_loudly(tmp_path):
    """No CPU fallback: loading a library that is not there raises, in a
    fresh interpreter (the module caches the loaded library)."""
    import subprocess
    import sys
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_1111_4971_gb300 import _lib\n"
        "try:\n"
        "    _lib.load(%r)\n"
        "except RuntimeError as e:\n"
        "    print('raised', 'no fallback' in str(e))\n"
        "else:\n"
        "    print('loaded')\n"
    ) % (str(__import__('pathlib').Path(__file__).resolve().parents[1]), str(tmp_path / "absent.so"))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert out.stdout.strip() == "raised True", out.stdout + out.stderr
