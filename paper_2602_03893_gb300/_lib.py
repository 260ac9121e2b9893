"""ctypes binding of libgpair.so (include/gpair.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Device memory and streams
come from PyTorch (CUDA tensors, torch.cuda streams); all computation runs in the library's
kernels.  There is no fallback: if the library cannot be loaded the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import build as _build

c_int, c_int64, c_float, c_void_p, c_double = ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p, ctypes.c_double

STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of device memory",
          4: "device-side wait timed out", 5: "unsupported shape or layout", 6: "non-finite input",
          7: "problem exceeds the fixed scratch of the allocation-free entry point"}

RULE_ADAM, RULE_GD_LINESEARCH = 0, 1
OP_EXACT, OP_ASSA = 0, 1          # gpair_step_params.op

# Symbols declared in include/gpair.h (checked by the CPU test suite).
EXPORTS = ("gpair_forward", "gpair_forward_noalloc", "gpair_adjoint", "gpair_shard_range", "gpair_forward_shard",
           "gpair_adjoint_shard", "gpair_voxelize", "gpair_solver_create", "gpair_solver_destroy",
           "gpair_step", "gpair_solver_image", "gpair_solver_get_state", "gpair_solver_set_state",
           "gpair_solver_profile", "gpair_solver_timings", "gpair_solver_steps",
           "gpair_reduce_f64", "gpair_status_string", "gpair_last_device_status", "gpair_release_scratch",
           "gpair_wait_selftest", "gpair_assa_forward", "gpair_assa_adjoint", "gpair_vcr", "gpair_zmap",
           "gpair_image_metrics", "gpair_pipe_peak", "gpair_version")


class GpairError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} failed: {STATUS.get(code, code)} ({code})")
        self.code = code


class _Grid(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("ox", c_float), ("oy", c_float), ("oz", c_float),
                ("dx", c_float), ("sigma", c_float)]


class _Gaussians(ctypes.Structure):
    _fields_ = [("M", c_int64), ("cx", c_void_p), ("cy", c_void_p), ("cz", c_void_p), ("sigma", c_void_p),
                ("A", c_void_p), ("grid", ctypes.POINTER(_Grid))]


class _Array(ctypes.Structure):
    _fields_ = [("n_sensors", c_int), ("xyz", c_void_p), ("sound_speed", c_float), ("fs", c_float),
                ("t0", c_float), ("n_samples", c_int), ("window_k", c_float)]


class _StepParams(ctypes.Structure):
    _fields_ = [("rule", c_int), ("npc", c_int), ("npc_eps", c_float), ("eta_max", c_float), ("eta_min", c_float),
                ("T0", c_int), ("T_mult", c_float), ("beta1", c_float), ("beta2", c_float), ("adam_eps", c_float),
                ("vcr_lambda", c_float), ("vcr_beta", c_float), ("vcr_eps", c_float), ("op", c_int), ("n_min", c_int)]


_lib = None


def load(path: str | None = None):
    """Load libgpair.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = path or _build.build()
        lib = ctypes.CDLL(path)
        P = c_void_p
        lib.gpair_forward.argtypes = [ctypes.POINTER(_Gaussians), ctypes.POINTER(_Array), P, P]
        lib.gpair_forward_noalloc.argtypes = [ctypes.POINTER(_Gaussians), ctypes.POINTER(_Array), P, P]
        lib.gpair_adjoint.argtypes = [ctypes.POINTER(_Gaussians), ctypes.POINTER(_Array), P, P, P, P, P]
        lib.gpair_shard_range.argtypes = [ctypes.POINTER(_Grid), c_int, c_int, ctypes.POINTER(c_int),
                                          ctypes.POINTER(c_int)]
        lib.gpair_forward_shard.argtypes = [ctypes.POINTER(_Gaussians), ctypes.POINTER(_Array), c_int, c_int, P, P]
        lib.gpair_adjoint_shard.argtypes = [ctypes.POINTER(_Gaussians), ctypes.POINTER(_Array), c_int, c_int, P, P, P]
        lib.gpair_voxelize.argtypes = [ctypes.POINTER(_Gaussians), ctypes.POINTER(_Grid), c_float, P, P]
        lib.gpair_solver_create.argtypes = [ctypes.POINTER(_Gaussians), ctypes.POINTER(_Array),
                                            ctypes.POINTER(_StepParams), ctypes.POINTER(c_void_p)]
        lib.gpair_solver_destroy.argtypes = [P]
        lib.gpair_solver_destroy.restype = None
        lib.gpair_step.argtypes = [P, P, ctypes.POINTER(c_double), ctypes.POINTER(c_double), P]
        lib.gpair_solver_steps.argtypes = [P, P, c_int, ctypes.POINTER(c_double), ctypes.POINTER(c_double), P]
        lib.gpair_solver_image.argtypes = [P, P, P]
        lib.gpair_solver_get_state.argtypes = [P, P, P, P, ctypes.POINTER(c_int), P]
        lib.gpair_solver_set_state.argtypes = [P, P, P, P, c_int, P]
        lib.gpair_solver_profile.argtypes = [P, c_int]
        lib.gpair_solver_timings.argtypes = [P, ctypes.POINTER(c_double), ctypes.POINTER(c_int)]
        lib.gpair_reduce_f64.argtypes = [P, P, P, c_int64, P, P]
        lib.gpair_status_string.argtypes = [c_int]
        lib.gpair_status_string.restype = ctypes.c_char_p
        lib.gpair_last_device_status.argtypes = [P]
        lib.gpair_release_scratch.argtypes = []
        lib.gpair_release_scratch.restype = None
        lib.gpair_wait_selftest.argtypes = [c_int, P]
        lib.gpair_pipe_peak.argtypes = [c_int, c_int, ctypes.POINTER(c_double), P]
        lib.gpair_assa_forward.argtypes = [P, P, c_int, P, P]
        lib.gpair_zmap.argtypes = [P, c_int, c_int, c_int, P, P]
        lib.gpair_image_metrics.argtypes = [P, P, c_int, c_int, c_int, c_int, c_float, ctypes.POINTER(c_double), P]
        lib.gpair_vcr.argtypes = [P, c_int, c_int, c_int, c_float, c_float, c_float, P, ctypes.POINTER(c_double), P]
        lib.gpair_assa_adjoint.argtypes = [P, P, c_int, P, P, P]
        lib.gpair_version.restype = ctypes.c_char_p
        _lib = lib
    return _lib


def library_path() -> str:
    return _build.LIB


# ---------------------------------------------------------------- Python-side descriptions

@dataclass
class Grid:
    """Grid of Gaussian centres (gpair_grid): centre of node idx is o + (idx + 1/2) dx, x fastest."""
    nx: int
    ny: int
    nz: int
    ox: float
    oy: float
    oz: float
    dx: float
    sigma: float

    def _c(self) -> _Grid:
        return _Grid(self.nx, self.ny, self.nz, self.ox, self.oy, self.oz, self.dx, self.sigma)


@dataclass
class Gaussians:
    """gpair_gaussians.  Grid-implicit (grid set, cx None) or SoA (cx, cy, cz, sigma set).
    All tensors: CUDA float32, contiguous, length M."""
    A: torch.Tensor
    grid: Grid | None = None
    cx: torch.Tensor | None = None
    cy: torch.Tensor | None = None
    cz: torch.Tensor | None = None
    sigma: torch.Tensor | None = None

    @property
    def M(self) -> int:
        return int(self.A.numel())

    def _c(self):
        keep = []
        g = _Gaussians()
        g.M = self.M
        g.A = _ptr(self.A)
        if self.cx is None:
            gr = self.grid._c()
            keep.append(gr)
            g.grid = ctypes.pointer(gr)
            g.cx = g.cy = g.cz = g.sigma = None
        else:
            g.cx, g.cy, g.cz, g.sigma = _ptr(self.cx), _ptr(self.cy), _ptr(self.cz), _ptr(self.sigma)
            g.grid = None
        return g, keep


@dataclass
class SensorArray:
    """gpair_array: sensors (CUDA float32 [Nd, 3]) and acquisition parameters."""
    xyz: torch.Tensor
    sound_speed: float
    fs: float
    n_samples: int
    t0: float = 0.0
    window_k: float = 3.0

    @property
    def n_sensors(self) -> int:
        return int(self.xyz.shape[0])

    def _c(self) -> _Array:
        return _Array(self.n_sensors, _ptr(self.xyz), self.sound_speed, self.fs, self.t0, self.n_samples,
                      self.window_k)


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if t.numel() and not t.is_cuda:
        raise ValueError("gpair expects CUDA tensors")
    if t.numel() and not t.is_contiguous():
        raise ValueError("gpair expects contiguous tensors")
    return t.data_ptr() if t.numel() else None


def _stream(stream):
    if stream is None:
        return c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return c_void_p(stream.cuda_stream)
    return c_void_p(int(stream))


def _check(name, code):
    if code != 0:
        raise GpairError(name, code)


# ---------------------------------------------------------------- entry points

def gpair_forward(g: Gaussians, arr: SensorArray, y: torch.Tensor, stream=None) -> torch.Tensor:
    lib = load()
    gc_, keep = g._c()
    ac = arr._c()
    _check("gpair_forward", lib.gpair_forward(ctypes.byref(gc_), ctypes.byref(ac), _ptr(y), _stream(stream)))
    return y


def gpair_forward_noalloc(g: Gaussians, arr: SensorArray, y: torch.Tensor, stream=None) -> torch.Tensor:
    """gpair_forward without any device allocation (fixed 64 MiB library-owned scratch; calls
    overlapping on the GPU race)."""
    lib = load()
    gc_, keep = g._c()
    ac = arr._c()
    _check("gpair_forward_noalloc", lib.gpair_forward_noalloc(ctypes.byref(gc_), ctypes.byref(ac), _ptr(y),
                                                              _stream(stream)))
    return y


def gpair_adjoint(g: Gaussians, arr: SensorArray, delta: torch.Tensor, gA: torch.Tensor,
                  gc: torch.Tensor | None = None, gsigma: torch.Tensor | None = None, stream=None):
    lib = load()
    gc_, keep = g._c()
    ac = arr._c()
    _check("gpair_adjoint", lib.gpair_adjoint(ctypes.byref(gc_), ctypes.byref(ac), _ptr(delta), _ptr(gA), _ptr(gc),
                                              _ptr(gsigma), _stream(stream)))
    return gA, gc, gsigma


def gpair_shard_range(grid: Grid, shard: int, n_shards: int):
    """Lattice rows [z_begin, z_end) of shard `shard` of `n_shards` (host arithmetic)."""
    zb, ze = c_int(0), c_int(0)
    gr = grid._c()
    _check("gpair_shard_range", load().gpair_shard_range(ctypes.byref(gr), int(shard), int(n_shards), ctypes.byref(zb),
                                                         ctypes.byref(ze)))
    return zb.value, ze.value


def gpair_forward_shard(g: Gaussians, arr: SensorArray, shard: int, n_shards: int, y: torch.Tensor,
                        stream=None) -> torch.Tensor:
    """Partial signals of the shard's z-slab of a grid-implicit set (they sum to gpair_forward)."""
    lib = load()
    gc_, keep = g._c()
    ac = arr._c()
    _check("gpair_forward_shard", lib.gpair_forward_shard(ctypes.byref(gc_), ctypes.byref(ac), int(shard),
                                                          int(n_shards), _ptr(y), _stream(stream)))
    return y


def gpair_adjoint_shard(g: Gaussians, arr: SensorArray, shard: int, n_shards: int, delta: torch.Tensor,
                        gA: torch.Tensor, stream=None) -> torch.Tensor:
    """Amplitude gradient of the shard's Gaussians (its rows of gA; the rest untouched)."""
    lib = load()
    gc_, keep = g._c()
    ac = arr._c()
    _check("gpair_adjoint_shard", lib.gpair_adjoint_shard(ctypes.byref(gc_), ctypes.byref(ac), int(shard),
                                                          int(n_shards), _ptr(delta), _ptr(gA), _stream(stream)))
    return gA


def gpair_assa_forward(g: Gaussians, arr: SensorArray, y: torch.Tensor, n_min: int = 25, stream=None) -> torch.Tensor:
    """The paper's discretised forward operator (adaptive supersampling alignment), grid Gaussians."""
    lib = load()
    gc_, keep = g._c()
    ac = arr._c()
    _check("gpair_assa_forward", lib.gpair_assa_forward(ctypes.byref(gc_), ctypes.byref(ac), int(n_min), _ptr(y),
                                                        _stream(stream)))
    return y


def gpair_assa_adjoint(g: Gaussians, arr: SensorArray, delta: torch.Tensor, gA: torch.Tensor, n_min: int = 25,
                       stream=None) -> torch.Tensor:
    """Transpose of gpair_assa_forward (amplitude gradient)."""
    lib = load()
    gc_, keep = g._c()
    ac = arr._c()
    _check("gpair_assa_adjoint", lib.gpair_assa_adjoint(ctypes.byref(gc_), ctypes.byref(ac), int(n_min), _ptr(delta),
                                                        _ptr(gA), _stream(stream)))
    return gA


def gpair_vcr(x: torch.Tensor, dims, beta: float, eps: float = 1e-8, lam: float = 1.0, grad: torch.Tensor | None = None,
              want_value: bool = True, stream=None):
    """Vessel continuity regulariser of a lattice image x (dims = (nz, ny, nx), x fastest):
    returns R_VCR(x) (FP64, synchronising) when want_value; adds lam * grad R_VCR into `grad`."""
    nz, ny, nx = dims
    val = c_double(0.0)
    _check("gpair_vcr", load().gpair_vcr(_ptr(x), int(nx), int(ny), int(nz), float(beta), float(eps), float(lam),
                                         _ptr(grad), ctypes.byref(val) if want_value else None, _stream(stream)))
    return val.value if want_value else None


def gpair_zmap(vol: torch.Tensor, dims, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Maximum amplitude projection along z of a (nz, ny, nx) volume."""
    nz, ny, nx = dims
    out = out if out is not None else torch.empty((ny, nx), device=vol.device, dtype=torch.float32)
    _check("gpair_zmap", load().gpair_zmap(_ptr(vol), nx, ny, nz, _ptr(out), _stream(stream)))
    return out


def gpair_image_metrics(x: torch.Tensor, ref: torch.Tensor, dims, win: int = 7, data_range: float = 1.0,
                        stream=None) -> dict:
    """MSE, PSNR (dB) and mean SSIM of x against ref; dims = (nz, ny, nx), nz = 1 for an image."""
    nz, ny, nx = dims
    out = (c_double * 3)()
    _check("gpair_image_metrics", load().gpair_image_metrics(_ptr(x), _ptr(ref), nx, ny, nz, int(win),
                                                             float(data_range), out, _stream(stream)))
    return {"mse": out[0], "psnr": out[1], "ssim": out[2]}


def gpair_voxelize(g: Gaussians, out_grid: Grid, window_k: float, vol: torch.Tensor, stream=None) -> torch.Tensor:
    lib = load()
    gc_, keep = g._c()
    og = out_grid._c()
    _check("gpair_voxelize", lib.gpair_voxelize(ctypes.byref(gc_), ctypes.byref(og), window_k, _ptr(vol),
                                                _stream(stream)))
    return vol


def gpair_reduce_f64(a, b, c, out, stream=None):
    lib = load()
    _check("gpair_reduce_f64", lib.gpair_reduce_f64(_ptr(a), _ptr(b), _ptr(c), a.numel(), _ptr(out), _stream(stream)))
    return out


def gpair_last_device_status(stream=None) -> int:
    return int(load().gpair_last_device_status(_stream(stream)))


def gpair_release_scratch() -> None:
    load().gpair_release_scratch()


def gpair_wait_selftest(polls: int, stream=None) -> None:
    """Launch the bounded-wait self-test (a wait nothing completes, given up after `polls` polls);
    the next gpair_last_device_status reports the timeout."""
    _check("gpair_wait_selftest", load().gpair_wait_selftest(int(polls), _stream(stream)))


PIPE_FP32, PIPE_MUFU = 0, 1


def gpair_pipe_peak(pipe: int, reps: int = 5, stream=None) -> float:
    """Measured lane operations per second of the FP32 FMA (PIPE_FP32) or MUFU ex2 (PIPE_MUFU)
    pipe on the current device."""
    out = c_double()
    _check("gpair_pipe_peak", load().gpair_pipe_peak(int(pipe), int(reps), ctypes.byref(out), _stream(stream)))
    return out.value


def gpair_version() -> str:
    return load().gpair_version().decode()


def gpair_status_string(code: int) -> str:
    return load().gpair_status_string(int(code)).decode()


@dataclass
class StepParams:
    rule: int = RULE_ADAM
    npc: int = 1
    npc_eps: float = 1e-8
    eta_max: float = 1e-2
    eta_min: float = 0.0
    T0: int = 20
    T_mult: float = 1.0
    beta1: float = 0.9
    beta2: float = 0.999
    adam_eps: float = 1e-8
    vcr_lambda: float = 0.0      # vessel continuity regulariser weight (0: off)
    vcr_beta: float = 0.0        # TV share of the regulariser
    vcr_eps: float = 1e-8
    op: int = OP_EXACT           # operator of the step's forwards and adjoints
    n_min: int = 25              # ASSA minimum pulse length (op = OP_ASSA)

    def _c(self) -> _StepParams:
        return _StepParams(self.rule, self.npc, self.npc_eps, self.eta_max, self.eta_min, self.T0, self.T_mult,
                           self.beta1, self.beta2, self.adam_eps, self.vcr_lambda, self.vcr_beta, self.vcr_eps,
                           self.op, self.n_min)


class Solver:
    """gpair_solver: Algorithm 2 on amplitudes (gpair_solver_create / gpair_step / ...).
    The geometry tensors of `g` must stay alive while the solver lives."""

    def __init__(self, g: Gaussians, arr: SensorArray, params: StepParams):
        lib = load()
        self._g, self._arr, self.params = g, arr, params
        gc_, self._keep = g._c()
        ac = arr._c()
        pc = params._c()
        h = c_void_p()
        _check("gpair_solver_create", lib.gpair_solver_create(ctypes.byref(gc_), ctypes.byref(ac), ctypes.byref(pc),
                                                              ctypes.byref(h)))
        self._h = h
        self.M = g.M

    def gpair_step(self, b: torch.Tensor, want_loss: bool = True, stream=None):
        lib = load()
        loss, resid = c_double(), c_double()
        _check("gpair_step", lib.gpair_step(self._h, _ptr(b), ctypes.byref(loss) if want_loss else None,
                                            ctypes.byref(resid) if want_loss else None, _stream(stream)))
        return (loss.value, resid.value) if want_loss else None

    def gpair_solver_steps(self, b: torch.Tensor, n: int, want_loss: bool = True, stream=None):
        """n steps replayed as one CUDA graph; (loss, resid) of the iterate entering the last one."""
        lib = load()
        loss, resid = c_double(), c_double()
        _check("gpair_solver_steps", lib.gpair_solver_steps(self._h, _ptr(b), int(n),
                                                            ctypes.byref(loss) if want_loss else None,
                                                            ctypes.byref(resid) if want_loss else None,
                                                            _stream(stream)))
        return (loss.value, resid.value) if want_loss else None

    def gpair_solver_image(self, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        out = out if out is not None else torch.empty(self.M, device="cuda", dtype=torch.float32)
        _check("gpair_solver_image", load().gpair_solver_image(self._h, _ptr(out), _stream(stream)))
        return out

    def gpair_solver_get_state(self, stream=None):
        z, m, v = (torch.empty(self.M, device="cuda", dtype=torch.float32) for _ in range(3))
        t = c_int()
        _check("gpair_solver_get_state", load().gpair_solver_get_state(self._h, _ptr(z), _ptr(m), _ptr(v),
                                                                       ctypes.byref(t), _stream(stream)))
        return z, m, v, t.value

    def gpair_solver_set_state(self, z=None, m=None, v=None, t: int = 0, stream=None):
        _check("gpair_solver_set_state", load().gpair_solver_set_state(self._h, _ptr(z), _ptr(m), _ptr(v), int(t),
                                                                       _stream(stream)))

    def gpair_solver_profile(self, enable: bool = True):
        _check("gpair_solver_profile", load().gpair_solver_profile(self._h, 1 if enable else 0))

    def gpair_solver_timings(self):
        """Summed device milliseconds (forward slab kernel, adjoint kernel, whole step) and the
        number of recorded steps."""
        ms = (c_double * 3)()
        n = c_int()
        _check("gpair_solver_timings", load().gpair_solver_timings(self._h, ms, ctypes.byref(n)))
        return list(ms), n.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().gpair_solver_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
