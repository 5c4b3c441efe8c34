"""FP64 CPU oracle for the pseudo-spectral Navier-Stokes hot path.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the bench's CPU
baseline leg use it; the product library never imports, links or runs it.

This module is a thin ctypes wrapper over ``ns_oracle.cpp`` (plain C++,
its own radix-2 FFT, no code shared with the CUDA path).  Every function takes
and returns numpy arrays in the canonical layouts described there:

* truncated spectral state, complex128: 3D ``(3, c, c, h)`` = (comp, kz, ky, kx),
  2D ``(c, h)`` = (ky, kx); ``kc = (N-1)//3``, ``c = 2 kc + 1``, ``h = kc + 1``;
  index ``i`` on a full axis holds ``k = i`` if ``i <= kc`` else ``i - c``.
* physical fields, float64: 3D ``(3, N, N, N)`` = (comp, z, y, x), 2D ``(N, N)``.

Parity status of each function is recorded in the tests that pin it
(``tests/test_oracle_*.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ns_oracle.cpp")
_LIB = os.path.join(_HERE, "libns_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libns_oracle.so`` (g++, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        sig = {
            "orc_threads": ([], I),
            "orc_set_threads": ([I], None),
            "orc_fft1d": ([P, I, I], I),
            "orc_rfftn": ([I, I, P, P], I),
            "orc_irfftn": ([I, I, P, P], I),
            "orc_phys_to_state": ([I, I, P, P], I),
            "orc_state_to_phys": ([I, I, P, P], I),
            "orc_rhs": ([I, I, P, P, P], I),
            "orc_rhs_modes": ([I, I, P, P, I, P, P], I),
            "orc_step": ([I, I, D, D, I, P, P], I),
            "orc_step_rk2": ([I, I, D, D, I, P, P], I),
            "orc_step_visc": ([I, I, D, D, D, D, I, I, P, P], I),
            "orc_velocity": ([I, I, P, P], I),
            "orc_step_cfl": ([I, I, D, D, D, I, I, P, P, P], I),
            "orc_diagnostics": ([I, I, P, ctypes.POINTER(D), ctypes.POINTER(D)], I),
            "orc_nbins": ([I, I], I),
            "orc_spectrum": ([I, I, P, P, I], I),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed (rc={rc})")


def sizes(n: int):
    """(kc, c, h) of the 2/3-rule truncation for N points per axis."""
    kc = (n - 1) // 3
    return kc, 2 * kc + 1, kc + 1


def state_shape(dim: int, n: int):
    _, c, h = sizes(n)
    return (3, c, c, h) if dim == 3 else (c, h)


def phys_shape(dim: int, n: int):
    return (3, n, n, n) if dim == 3 else (n, n)


def threads() -> int:
    return _load().orc_threads()


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def fft1d(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised 1D DFT, ``X_k = sum_j x_j exp(sign 2 pi i j k / n)``."""
    y = np.ascontiguousarray(x, dtype=np.complex128).copy()
    _check(_load().orc_fft1d(_ptr(y), y.size, int(sign)), "fft1d")
    return y


def rfftn(dim: int, n: int, phys: np.ndarray) -> np.ndarray:
    p = np.ascontiguousarray(phys, dtype=np.float64)
    shape = (n, n, n // 2 + 1) if dim == 3 else (n, n // 2 + 1)
    out = np.zeros(shape, np.complex128)
    _check(_load().orc_rfftn(dim, n, _ptr(p), _ptr(out)), "rfftn")
    return out


def irfftn(dim: int, n: int, spec: np.ndarray) -> np.ndarray:
    s = np.ascontiguousarray(spec, dtype=np.complex128)
    out = np.zeros((n,) * dim, np.float64)
    _check(_load().orc_irfftn(dim, n, _ptr(s), _ptr(out)), "irfftn")
    return out


def phys_to_state(dim: int, n: int, phys: np.ndarray) -> np.ndarray:
    p = np.ascontiguousarray(phys, dtype=np.float64).reshape(phys_shape(dim, n))
    out = np.zeros(state_shape(dim, n), np.complex128)
    _check(_load().orc_phys_to_state(dim, n, _ptr(p), _ptr(out)), "phys_to_state")
    return out


def state_to_phys(dim: int, n: int, state: np.ndarray) -> np.ndarray:
    s = np.ascontiguousarray(state, dtype=np.complex128).reshape(state_shape(dim, n))
    out = np.zeros(phys_shape(dim, n), np.float64)
    _check(_load().orc_state_to_phys(dim, n, _ptr(s), _ptr(out)), "state_to_phys")
    return out


def rhs(dim: int, n: int, state: np.ndarray, forcing: np.ndarray | None = None) -> np.ndarray:
    s = np.ascontiguousarray(state, dtype=np.complex128).reshape(state_shape(dim, n))
    f = None if forcing is None else np.ascontiguousarray(forcing, dtype=np.complex128).reshape(s.shape)
    out = np.zeros_like(s)
    _check(_load().orc_rhs(dim, n, _ptr(s), None if f is None else _ptr(f), _ptr(out)), "rhs")
    return out


def rhs_modes(n: int, state: np.ndarray, modes, forcing: np.ndarray | None = None) -> np.ndarray:
    """Nonlinear term of the 3D state on selected modes by the direct Galerkin
    sum over retained triads (no FFT): ``modes`` is a sequence of (kx, ky, kz)
    with 0 <= kx <= kc, |ky|, |kz| <= kc; returns complex128 ``(len(modes), 3)``.
    About c^3 triads per mode (c = 2 kc + 1), spread over the oracle's threads."""
    s = np.ascontiguousarray(state, dtype=np.complex128).reshape(state_shape(3, n))
    f = None if forcing is None else np.ascontiguousarray(forcing, dtype=np.complex128).reshape(s.shape)
    k = np.ascontiguousarray(np.asarray(modes, dtype=np.int32).reshape(-1, 3))
    out = np.zeros((k.shape[0], 3), np.complex128)
    _check(_load().orc_rhs_modes(3, n, _ptr(s), None if f is None else _ptr(f), int(k.shape[0]), _ptr(k),
                                 _ptr(out)), "rhs_modes")
    return out


def step(dim: int, n: int, nu: float, dt: float, nsteps: int, state: np.ndarray,
         forcing: np.ndarray | None = None, order: int = 4, nu4: float = 0.0, nu8: float = 0.0) -> np.ndarray:
    """Return the state after ``nsteps`` Lawson IF-RK steps of the given order
    (4, or 2 = the midpoint form) with the damping rate
    nu |k|^2 + nu4 |k|^4 + nu8 |k|^8 (input untouched)."""
    s = np.ascontiguousarray(state, dtype=np.complex128).reshape(state_shape(dim, n)).copy()
    f = None if forcing is None else np.ascontiguousarray(forcing, dtype=np.complex128).reshape(s.shape)
    _check(_load().orc_step_visc(dim, n, float(nu), float(nu4), float(nu8), float(dt), int(order), int(nsteps),
                                 None if f is None else _ptr(f), _ptr(s)), "step")
    return s


def velocity(dim: int, n: int, state: np.ndarray) -> np.ndarray:
    """Physical velocity ``(dim, N, ..)`` of a state (2D: from the stream function)."""
    s = np.ascontiguousarray(state, dtype=np.complex128).reshape(state_shape(dim, n))
    out = np.empty((dim,) + (n,) * dim, np.float64)
    _check(_load().orc_velocity(dim, n, _ptr(s), _ptr(out)), "velocity")
    return out


def step_cfl(dim: int, n: int, nu: float, dt_max: float, cfl: float, nsteps: int, state: np.ndarray,
             forcing: np.ndarray | None = None, order: int = 4):
    """(state, dts) after ``nsteps`` steps whose dt follows the CFL rule
    dt = min(dt_max, cfl * min_i (2 pi / N) / max|u_i|), chosen before each step."""
    s = np.ascontiguousarray(state, dtype=np.complex128).reshape(state_shape(dim, n)).copy()
    f = None if forcing is None else np.ascontiguousarray(forcing, dtype=np.complex128).reshape(s.shape)
    dts = np.zeros(max(int(nsteps), 1), np.float64)
    _check(_load().orc_step_cfl(dim, n, float(nu), float(dt_max), float(cfl), int(order), int(nsteps),
                                None if f is None else _ptr(f), _ptr(s), _ptr(dts)), "step_cfl")
    return s, dts[:nsteps]


def diagnostics(dim: int, n: int, state: np.ndarray):
    s = np.ascontiguousarray(state, dtype=np.complex128).reshape(state_shape(dim, n))
    e = ctypes.c_double()
    o = ctypes.c_double()
    _check(_load().orc_diagnostics(dim, n, _ptr(s), ctypes.byref(e), ctypes.byref(o)), "diagnostics")
    return e.value, o.value


def nbins(dim: int, n: int) -> int:
    return _load().orc_nbins(dim, n)


def spectrum(dim: int, n: int, state: np.ndarray) -> np.ndarray:
    s = np.ascontiguousarray(state, dtype=np.complex128).reshape(state_shape(dim, n))
    nb = nbins(dim, n)
    out = np.zeros(nb, np.float64)
    _check(_load().orc_spectrum(dim, n, _ptr(s), _ptr(out), nb), "spectrum")
    return out


def _wavevectors(dim: int, n: int):
    """Integer wavevector components on the truncated layout, broadcastable to
    the state's spectral shape (without the component axis)."""
    kc, c, h = sizes(n)
    i = np.arange(c)
    kfull = np.where(i <= kc, i, i - c)
    if dim == 2:
        return np.arange(h)[None, :], kfull[:, None], np.zeros((1, 1), dtype=np.int64)
    return np.arange(h)[None, None, :], kfull[None, :, None], kfull[:, None, None]


def budget(dim: int, n: int, nu: float, state: np.ndarray, forcing: np.ndarray | None = None,
           nu4: float = 0.0, nu8: float = 0.0):
    """Energy and enstrophy budget terms (P_E, D_E, P_Z, D_Z) of a truncated
    spectral state: forcing power and dissipation, the "spatial means" of the
    paper's output list besides energy and enstrophy.  With the mode weights
    w = 1 on kx = 0 and 2 elsewhere (the half spectrum stands for the full one)
    and the damping rate d = nu k^2 + nu4 k^4 + nu8 k^8 of a mode:
    3D velocity:  P_E = sum w Re(u* . F), D_E = sum w d |u|^2,
                  P_Z = sum w k^2 Re(u* . F), D_Z = sum w k^2 d |u|^2;
    2D vorticity: P_E = sum w Re(w* F) / k^2, D_E = sum w d |w|^2 / k^2,
                  P_Z = sum w Re(w* F), D_Z = sum w d |w|^2  (k = 0 excluded).
    Plain numpy in float64 (no FFT involved)."""
    s = np.ascontiguousarray(state, dtype=np.complex128).reshape(state_shape(dim, n))
    f = np.zeros_like(s) if forcing is None else np.ascontiguousarray(forcing, dtype=np.complex128).reshape(s.shape)
    kx, ky, kz = _wavevectors(dim, n)
    k2 = (kx * kx + ky * ky + kz * kz).astype(np.float64)
    w = np.where(kx == 0, 1.0, 2.0) * np.ones_like(k2)
    d = nu * k2 + nu4 * k2 ** 2 + nu8 * k2 ** 4
    if dim == 3:
        m2 = np.sum(np.abs(s) ** 2, axis=0)
        pf = np.sum((np.conj(s) * f).real, axis=0)
        return (float(np.sum(w * pf)), float(np.sum(w * d * m2)),
                float(np.sum(w * k2 * pf)), float(np.sum(w * k2 * d * m2)))
    m2 = np.abs(s) ** 2
    pf = (np.conj(s) * f).real
    nz = k2 > 0
    inv = np.where(nz, 1.0 / np.where(nz, k2, 1.0), 0.0)
    return (float(np.sum(w * pf * inv)), float(np.sum(w * d * inv * m2)),
            float(np.sum(w * pf * nz)), float(np.sum(w * d * m2)))
