"""CPU checks of the boundary: the library builds, loads and exports every entry point that
include/gpair.h declares; host-side argument validation rejects bad input without touching
the GPU; the product path has no fallback to the oracle."""
import ctypes
import os
import re

import pytest

from paper_2602_03893_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header=None):
    inc = os.path.join(ROOT, "include")
    names = set()
    for h in sorted(os.listdir(inc)):
        if not h.endswith(".h") or (header and h != header):
            continue
        src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, h)).read(), flags=re.S)
        names |= set(re.findall(r"\b(gpair_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declarations_are_all_exported(lib):
    names = declared_functions()
    assert "gpair_forward" in names and "gpair_adjoint" in names and "gpair_step" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/*.h but not exported"
    assert set(_lib.EXPORTS) == set(declared_functions("gpair.h"))
    assert "gpair_conv3d_fwd" in names and "gpair_conv3d_wgrad" in names


def test_status_strings_and_version(lib):
    lib.gpair_status_string.restype = ctypes.c_char_p
    lib.gpair_version.restype = ctypes.c_char_p
    assert lib.gpair_status_string(0) == b"ok"
    assert b"invalid" in lib.gpair_status_string(1)
    assert b"sm_103a" in lib.gpair_version()


def test_invalid_arguments_rejected_before_any_launch(lib):
    """Validation runs on the host: NULL structs and non-positive sizes return INVALID_ARG (1)
    without a CUDA call, so this works without a GPU."""
    lib.gpair_forward.argtypes = [ctypes.c_void_p] * 4
    assert lib.gpair_forward(None, None, None, None) == 1
    g = _lib._Gaussians()
    g.M = 0
    a = _lib._Array()
    assert lib.gpair_forward(ctypes.byref(g), ctypes.byref(a), None, None) == 1
    grid = _lib._Grid(4, 4, 4, 0.0, 0.0, 0.0, 1e-4, 1e-4)
    g.M = 63                       # inconsistent with 4x4x4
    g.A = 1024                     # never dereferenced on this path
    g.grid = ctypes.pointer(grid)
    a.n_sensors, a.xyz, a.sound_speed, a.fs, a.n_samples, a.window_k = 1, 1024, 1500.0, 40e6, 16, 3.0
    assert lib.gpair_forward(ctypes.byref(g), ctypes.byref(a), ctypes.c_void_p(1024), None) == 1
    g.M = 64
    a.fs = -1.0
    assert lib.gpair_forward(ctypes.byref(g), ctypes.byref(a), ctypes.c_void_p(1024), None) == 1
    a.fs = 40e6
    a.window_k = 0.0
    assert lib.gpair_forward(ctypes.byref(g), ctypes.byref(a), ctypes.c_void_p(1024), None) == 1


def test_size_limits_and_new_entry_points_rejected_on_the_host(lib):
    """The documented limits (N_t <= 2^27, N_d <= 65535) and the argument checks of the ASSA,
    regulariser and metric entry points return their status before any CUDA call."""
    grid = _lib._Grid(4, 4, 4, 0.0, 0.0, 0.0, 1e-4, 1e-4)
    g = _lib._Gaussians()
    g.M, g.A, g.grid = 64, 1024, ctypes.pointer(grid)
    a = _lib._Array()
    a.n_sensors, a.xyz, a.sound_speed, a.fs, a.n_samples, a.window_k = 1, 1024, 1500.0, 40e6, 16, 3.0
    y = ctypes.c_void_p(1024)
    a.n_samples = (1 << 27) + 1
    assert lib.gpair_forward(ctypes.byref(g), ctypes.byref(a), y, None) == 5
    a.n_samples, a.n_sensors = 16, 65536
    assert lib.gpair_forward(ctypes.byref(g), ctypes.byref(a), y, None) == 5
    a.n_sensors = 1
    lib.gpair_assa_forward.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.gpair_assa_forward(ctypes.byref(g), ctypes.byref(a), 0, y, None) == 1          # n_min < 1
    soa = _lib._Gaussians()
    soa.M, soa.A, soa.cx, soa.cy, soa.cz, soa.sigma = 64, 1024, 1024, 1024, 1024, 1024
    assert lib.gpair_assa_forward(ctypes.byref(soa), ctypes.byref(a), 25, y, None) == 5      # one width needed
    lib.gpair_vcr.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                              ctypes.c_float, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.gpair_vcr(y, 0, 4, 4, 0.5, 1e-8, 1.0, None, None, None) == 1
    assert lib.gpair_vcr(y, 4, 4, 4, 0.5, -1.0, 1.0, None, None, None) == 1
    lib.gpair_image_metrics.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]
    out = (ctypes.c_double * 3)()
    assert lib.gpair_image_metrics(y, y, 8, 8, 8, 4, 1.0, out, None) == 1                      # even window
    assert lib.gpair_image_metrics(y, y, 8, 8, 5, 7, 1.0, out, None) == 5                      # z shorter than it
    lib.gpair_wait_selftest.argtypes = [ctypes.c_int, ctypes.c_void_p]
    assert lib.gpair_wait_selftest(0, None) == 1
    # solver operator choice: op outside {0, 1}, n_min < 1 and free centres with ASSA
    lib.gpair_solver_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    h = ctypes.c_void_p()
    prm = _lib.StepParams(op=2)._c()
    assert lib.gpair_solver_create(ctypes.byref(g), ctypes.byref(a), ctypes.byref(prm), ctypes.byref(h)) == 1
    prm = _lib.StepParams(op=_lib.OP_ASSA, n_min=0)._c()
    assert lib.gpair_solver_create(ctypes.byref(g), ctypes.byref(a), ctypes.byref(prm), ctypes.byref(h)) == 1
    prm = _lib.StepParams(op=_lib.OP_ASSA)._c()
    assert lib.gpair_solver_create(ctypes.byref(soa), ctypes.byref(a), ctypes.byref(prm), ctypes.byref(h)) == 5
    assert not h
    lib.gpair_solver_steps.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]
    assert lib.gpair_solver_steps(None, y, 3, None, None, None) == 1                        # no solver
    lib.gpair_pipe_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    rate = ctypes.c_double()
    assert lib.gpair_pipe_peak(2, 5, ctypes.byref(rate), None) == 1                            # unknown pipe
    assert lib.gpair_pipe_peak(0, 0, ctypes.byref(rate), None) == 1                            # reps < 1
    assert lib.gpair_pipe_peak(0, 5, None, None) == 1


def test_product_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2602_03893_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "gpair_oracle" not in txt, f
