"""FP64 CPU oracle for the GPAIR forward/adjoint hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` leg and
``--impl reference``) may import this package.  It wraps ``gpair_oracle.c`` (plain C, FP64,
OpenMP over independent outputs) through ctypes and shares nothing with the CUDA library.

Every function takes float arrays exactly as the CUDA path receives them and converts them to
float64 here; results are float64.  Section/equation citations are in ``gpair_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gpair_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgpair_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gpair_oracle.c into oracle/_build/libgpair_oracle.so (gcc, -O2, OpenMP, no FMA
    contraction so every double operation rounds as written)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        _lib.ora_sphere_integral.restype = f64
        _lib.ora_sphere_integral.argtypes = [f64, f64, f64, f64]
        _lib.ora_pressure_exact.restype = f64
        _lib.ora_pressure_exact.argtypes = [f64, f64, f64, f64, f64]
        _lib.ora_pressure_outgoing.restype = f64
        _lib.ora_pressure_outgoing.argtypes = [f64, f64, f64, f64, f64]
        _lib.ora_forward.restype = None
        _lib.ora_forward.argtypes = [i64, dp, dp, dp, dp, dp, i32, dp, f64, f64, f64, i32,
                                     f64, i32, f64, dp, dp]
        _lib.ora_adjoint.restype = None
        _lib.ora_adjoint.argtypes = [i64, dp, dp, dp, dp, dp, i32, dp, f64, f64, f64, i32,
                                     f64, dp, f64, dp, dp, dp, dp, dp, dp, dp, dp]
        _lib.ora_voxelize.restype = None
        _lib.ora_voxelize.argtypes = [i64, dp, dp, dp, dp, dp, f64, i32, i32, i32,
                                      f64, f64, f64, f64, dp]
        _lib.ora_cawr.restype = f64
        _lib.ora_cawr.argtypes = [i32, f64, f64, i32, f64]
        _lib.ora_adam.restype = None
        _lib.ora_adam.argtypes = [i64, dp, dp, dp, dp, i32, f64, f64, f64, f64]
        _lib.ora_ir.restype = None
        _lib.ora_ir.argtypes = [i64, dp, dp, dp, dp, i32, dp, f64, f64, f64, i32, f64,
                                dp, i32, i32, i32, f64, f64, f64, i32, f64, f64, f64, f64,
                                dp, dp, dp]
        _lib.ora_assa_params.restype = None
        ip = ctypes.POINTER(ctypes.c_int)
        _lib.ora_assa_params.argtypes = [f64, f64, f64, i32, ip, ip, ip]
        _lib.ora_assa_forward.restype = None
        _lib.ora_assa_forward.argtypes = [i64, dp, dp, dp, dp, f64, i32, dp, f64, f64, f64, i32, i32, f64,
                                          dp, dp]
        _lib.ora_assa_adjoint.restype = None
        _lib.ora_assa_adjoint.argtypes = [i64, dp, dp, dp, f64, i32, dp, f64, f64, f64, i32, i32, dp, f64,
                                          dp, dp]
        _lib.ora_set_threads.argtypes = [i32]
        _lib.ora_get_threads.restype = i32
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n: int) -> None:
    _load().ora_set_threads(int(n))


def get_threads() -> int:
    return int(_load().ora_get_threads())


@dataclass
class Gaussians:
    """Explicit Gaussian set in float64: centres (M,3), sigma (M,), amplitude (M,)."""
    c: np.ndarray
    sigma: np.ndarray
    A: np.ndarray

    @property
    def M(self) -> int:
        return int(self.A.shape[0])


def gaussians_from_grid(nx, ny, nz, ox, oy, oz, h, sigma, A) -> Gaussians:
    """Grid-implicit Gaussian set (Methods, GKD: one Gaussian per voxel centre): centre of
    voxel (ix, iy, iz) is o + (idx + 1/2) h, x fastest; every Gaussian has width sigma.  The
    float32 grid parameters are widened exactly to float64 before use."""
    f = lambda q: float(np.float32(q))
    ox, oy, oz, h, sigma = f(ox), f(oy), f(oz), f(h), f(sigma)
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    c = np.stack([ox + (ix.ravel() + 0.5) * h, oy + (iy.ravel() + 0.5) * h,
                  oz + (iz.ravel() + 0.5) * h], axis=1)
    M = nx * ny * nz
    return Gaussians(c=c, sigma=np.full(M, sigma), A=_d(A).ravel().copy())


def gaussians_from_soa(cx, cy, cz, sigma, A) -> Gaussians:
    return Gaussians(c=np.stack([_d(cx), _d(cy), _d(cz)], axis=1), sigma=_d(sigma).copy(), A=_d(A).copy())


def sphere_integral(A, sigma, r, rp) -> float:
    return _load().ora_sphere_integral(A, sigma, r, rp)


def pressure_exact(A, sigma, r, t, v) -> float:
    return _load().ora_pressure_exact(A, sigma, r, t, v)


def pressure_outgoing(A, sigma, r, t, v) -> float:
    return _load().ora_pressure_outgoing(A, sigma, r, t, v)


def forward(g: Gaussians, sensors, v, fs, t0, Nt, k=3.0, mode="windowed", tau=0.0,
            want_amb=False, A=None):
    """Forward operator (Eq. single_forward summed over Gaussians; see ora_forward).
    Returns y (Nd, Nt) float64, or (y, amb) when want_amb."""
    lib = _load()
    s = _d(sensors).reshape(-1, 3)
    Nd = s.shape[0]
    cx, cy, cz = (_d(g.c[:, q]) for q in range(3))
    sg = _d(g.sigma)
    Aa = _d(g.A if A is None else A)
    y = np.zeros((Nd, Nt))
    amb = np.zeros((Nd, Nt)) if want_amb else None
    lib.ora_forward(g.M, _p(cx), _p(cy), _p(cz), _p(sg), _p(Aa), Nd, _p(s), float(v), float(fs),
                    float(t0), int(Nt), float(k), 0 if mode == "windowed" else 1, float(tau),
                    _p(y), _p(amb))
    return (y, amb) if want_amb else y


def adjoint(g: Gaussians, sensors, v, fs, t0, Nt, delta, k=3.0, want=("A",), tau=0.0,
            want_amb=False):
    """Adjoint of the windowed forward and the closed-form c / sigma gradients (ora_adjoint).
    want: subset of ("A", "c", "sigma").  Returns dict of float64 arrays (gc is (3, M)); with
    want_amb also "ambA", "ambC", "ambS"."""
    lib = _load()
    s = _d(sensors).reshape(-1, 3)
    Nd = s.shape[0]
    M = g.M
    cx, cy, cz = (_d(g.c[:, q]) for q in range(3))
    sg, Aa = _d(g.sigma), _d(g.A)
    dl = _d(delta).reshape(Nd, Nt)
    out = {}
    gA = np.zeros(M) if "A" in want else None
    gc = np.zeros((3, M)) if "c" in want else None
    gs = np.zeros(M) if "sigma" in want else None
    amb = [np.zeros(M) for _ in range(3)] if want_amb else [None, None, None]
    gcx, gcy, gcz = (None, None, None) if gc is None else (gc[0], gc[1], gc[2])
    lib.ora_adjoint(M, _p(cx), _p(cy), _p(cz), _p(sg), _p(Aa), Nd, _p(s), float(v), float(fs),
                    float(t0), int(Nt), float(k), _p(dl), float(tau), _p(gA), _p(gcx), _p(gcy),
                    _p(gcz), _p(gs), _p(amb[0]), _p(amb[1]), _p(amb[2]))
    if gA is not None:
        out["A"] = gA
    if gc is not None:
        out["c"] = gc
    if gs is not None:
        out["sigma"] = gs
    if want_amb:
        out["ambA"], out["ambC"], out["ambS"] = amb
    return out


def assa_params(sigma, v, fs, n_min=25):
    """(N_half, alpha, K) of the ASSA grid (ora_assa_params)."""
    nh, a, K = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _load().ora_assa_params(float(sigma), float(v), float(fs), int(n_min), ctypes.byref(nh), ctypes.byref(a),
                            ctypes.byref(K))
    return nh.value, a.value, K.value


def assa_forward(g: Gaussians, sigma, sensors, v, fs, t0, Nt, n_min=25, tau=0.0, want_amb=False):
    """ASSA forward (Algorithm 1, ForwardOp) for Gaussians sharing the width sigma.
    Returns y (Nd, Nt), or (y, amb) when want_amb."""
    lib = _load()
    s = _d(sensors).reshape(-1, 3)
    Nd = s.shape[0]
    cx, cy, cz = (_d(g.c[:, q]) for q in range(3))
    y = np.zeros((Nd, Nt))
    amb = np.zeros((Nd, Nt)) if want_amb else None
    lib.ora_assa_forward(g.M, _p(cx), _p(cy), _p(cz), _p(_d(g.A)), float(sigma), Nd, _p(s), float(v), float(fs),
                         float(t0), int(Nt), int(n_min), float(tau), _p(y), _p(amb))
    return (y, amb) if want_amb else y


def assa_adjoint(g: Gaussians, sigma, sensors, v, fs, t0, Nt, delta, n_min=25, tau=0.0, want_amb=False):
    """ASSA adjoint (Algorithm 1, AdjointOp): g (M,), or (g, amb) when want_amb."""
    lib = _load()
    s = _d(sensors).reshape(-1, 3)
    Nd = s.shape[0]
    cx, cy, cz = (_d(g.c[:, q]) for q in range(3))
    dl = _d(delta).reshape(Nd, Nt)
    gA = np.zeros(g.M)
    amb = np.zeros(g.M) if want_amb else None
    lib.ora_assa_adjoint(g.M, _p(cx), _p(cy), _p(cz), float(sigma), Nd, _p(s), float(v), float(fs), float(t0),
                         int(Nt), int(n_min), _p(dl), float(tau), _p(gA), _p(amb))
    return (gA, amb) if want_amb else gA


def voxelize(g: Gaussians, k, nx, ny, nz, ox, oy, oz, h):
    """Eq. (2) sampled at voxel centres, box-truncated at k sigma per axis (ora_voxelize).
    Returns (nz, ny, nx) float64."""
    lib = _load()
    cx, cy, cz = (_d(g.c[:, q]) for q in range(3))
    vol = np.zeros((nz, ny, nx))
    f = lambda q: float(np.float32(q))
    lib.ora_voxelize(g.M, _p(cx), _p(cy), _p(cz), _p(_d(g.sigma)), _p(_d(g.A)), float(k),
                     nx, ny, nz, f(ox), f(oy), f(oz), f(h), _p(vol))
    return vol


def cawr(t, eta_max, eta_min, T0, Tmult=1.0) -> float:
    return _load().ora_cawr(int(t), float(eta_max), float(eta_min), int(T0), float(Tmult))


def adam(z, m, v, g, t, eta, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam update of float64 arrays z, m, v with gradient g at step t (>= 1)."""
    for a in (z, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    gg = _d(g)
    _load().ora_adam(z.size, _p(z), _p(m), _p(v), _p(gg), int(t), float(eta), float(b1),
                     float(b2), float(eps))


def ir(g: Gaussians, sensors, v, fs, t0, Nt, b, iters, k=3.0, rule="adam", npc=True,
       npc_eps=1e-8, eta_max=1e-2, eta_min=0.0, T0=None, Tmult=1.0, b1=0.9, b2=0.999,
       adam_eps=1e-8):
    """Algorithm 2 on amplitudes (ora_ir).  Returns (x*, loss[iters], resid[iters])."""
    lib = _load()
    s = _d(sensors).reshape(-1, 3)
    Nd = s.shape[0]
    cx, cy, cz = (_d(g.c[:, q]) for q in range(3))
    bb = _d(b).reshape(Nd, Nt)
    x = np.zeros(g.M)
    loss = np.zeros(iters)
    resid = np.zeros(iters)
    lib.ora_ir(g.M, _p(cx), _p(cy), _p(cz), _p(_d(g.sigma)), Nd, _p(s), float(v), float(fs),
               float(t0), int(Nt), float(k), _p(bb), int(iters), 0 if rule == "adam" else 1,
               1 if npc else 0, float(npc_eps), float(eta_max), float(eta_min),
               int(T0 if T0 is not None else iters), float(Tmult), float(b1), float(b2),
               float(adam_eps), _p(x), _p(loss), _p(resid))
    return x, loss, resid


def ir_assa(g: Gaussians, sigma, sensors, v, fs, t0, Nt, b, iters, n_min=25, rule="adam", npc=True,
            npc_eps=1e-8, eta_max=1e-2, eta_min=0.0, T0=None, Tmult=1.0, b1=0.9, b2=0.999, adam_eps=1e-8):
    """Algorithm 2 on amplitudes with the paper's discretised operator (Algorithm 1) as F and F^T:
    the same iteration as `ir` (NPC x = (z + eps)^2, L = |F x - b|^2 / N, exact gradient
    F^T (2 (y - b) / N) chained through NPC, CAWR step size, Adam; or steepest descent with the
    exact line search alpha = <r, F g> / |F g|^2), for Gaussians sharing the width sigma.
    Returns (x*, loss[iters], resid[iters]) for the iterate entering each iteration."""
    s = _d(sensors).reshape(-1, 3)
    Nd = s.shape[0]
    bb = _d(b).reshape(Nd, Nt)
    N = float(Nd * Nt)
    z, m, vv = np.zeros(g.M), np.zeros(g.M), np.zeros(g.M)
    loss, resid = np.zeros(iters), np.zeros(iters)
    F = lambda x: assa_forward(Gaussians(g.c, g.sigma, x), sigma, s, v, fs, t0, Nt, n_min=n_min)
    Ft = lambda d: assa_adjoint(g, sigma, s, v, fs, t0, Nt, d, n_min=n_min)
    T0 = T0 if T0 is not None else iters
    for t in range(iters):
        x = (z + npc_eps) ** 2 if (npc and rule == "adam") else z.copy()
        r = F(x) - bb
        ss = float(np.sum(r * r))
        loss[t], resid[t] = ss / N, np.sqrt(ss)
        if rule == "adam":
            gz = Ft(2.0 * r / N)
            if npc:
                gz = gz * 2.0 * (z + npc_eps)
            adam(z, m, vv, np.ascontiguousarray(gz), t + 1, cawr(t, eta_max, eta_min, T0, Tmult), b1, b2,
                 adam_eps)
        else:
            gg = Ft(r)
            Fg = F(gg)
            den = float(np.sum(Fg * Fg))
            z -= (float(np.sum(r * Fg)) / den if den > 0.0 else 0.0) * gg
    x = (z + npc_eps) ** 2 if (npc and rule == "adam") else z
    return x, loss, resid
