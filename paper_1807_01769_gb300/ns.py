"""Thin ctypes binding of libns_gb300.so (C ABI in include/ns.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  The module-level functions carry the C names; ``Solver`` is a
small convenience wrapper over them.  Importing this module loads the
library and raises if it is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libns_gb300.so")

NS_OK = 0
NS_EINVAL = -1
NS_ENOMEM = -2
NS_ECUDA = -3
NS_EUNSUPPORTED = -4
NS_ENONFINITE = -5
NS_ETIMEOUT = -6
NS_FP64 = 0
NS_FP32 = 1
NS_FP32_TC = 2

ERROR_NAMES = {0: "NS_OK", -1: "NS_EINVAL", -2: "NS_ENOMEM", -3: "NS_ECUDA", -4: "NS_EUNSUPPORTED",
               -5: "NS_ENONFINITE", -6: "NS_ETIMEOUT"}


class ns_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("precision", ctypes.c_int)]


# (name, argtypes, restype) of every exported symbol declared in include/ns.h
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_LL = ctypes.c_longlong
_PI = ctypes.POINTER(ctypes.c_int)
_PD = ctypes.POINTER(ctypes.c_double)
_PLL = ctypes.POINTER(ctypes.c_longlong)
SIGNATURES = {
    "ns_sizes": ([ctypes.POINTER(ns_grid), _PI, _PI, _PI, _PLL, _PLL, _PI], _I),
    "ns_init": ([ctypes.POINTER(_P), ctypes.POINTER(ns_grid), _D, _D, _P], _I),
    "ns_set_state": ([_P, _P], _I),
    "ns_get_state": ([_P, _P], _I),
    "ns_set_state_spectral": ([_P, _P], _I),
    "ns_get_state_spectral": ([_P, _P], _I),
    "ns_step": ([_P, _I], _I),
    "ns_eval_rhs": ([_P, _P], _I),
    "ns_diagnostics": ([_P, _PD, _PD], _I),
    "ns_energy_spectrum": ([_P, _P, _PI], _I),
    "ns_set_stream": ([_P, _P], _I),
    "ns_sync": ([_P], _I),
    "ns_profile_step": ([_P, _I, _P, _P, _I], _I),
    "ns_num_kernels": ([], _I),
    "ns_kernel_name": ([_I], ctypes.c_char_p),
    "ns_kernel_bytes": ([_P, _I], _LL),
    "ns_device_bytes": ([_P], _LL),
    "ns_diagnostics_noalloc": ([ctypes.POINTER(ns_grid), _P, _P, _P], _I),
    "ns_fp32_fma_peak": ([_I, _PD], _I),
    "ns_destroy": ([_P], None),
    "ns_last_error": ([_P], ctypes.c_char_p),
    "ns_ensemble_init": ([ctypes.POINTER(_P), _I, _P, _I, _D, _D, _I], _I),
    "ns_ensemble_schedule": ([_P, _PI, _PI, _PI], _I),
    "ns_ensemble_set_schedule": ([_P, _I, _I, _I], _I),
    "ns_ensemble_tiles": ([_P, _PI, _PI], _I),
    "ns_ensemble_set_tiles": ([_P, _I, _I], _I),
    "ns_ensemble_fused": ([_P, _PI, _PI], _I),
    "ns_ensemble_set_fused": ([_P, _I], _I),
    "ns_ensemble_set_state_spectral": ([_P, _I, _P], _I),
    "ns_ensemble_get_state_spectral": ([_P, _I, _P], _I),
    "ns_ensemble_step": ([_P, _I], _I),
    "ns_ensemble_diagnostics": ([_P, _P, _P], _I),
    "ns_ensemble_set_stream": ([_P, _P], _I),
    "ns_ensemble_sync": ([_P], _I),
    "ns_ensemble_destroy": ([_P], None),
    "ns_ensemble_last_error": ([_P], ctypes.c_char_p),
    "ns_budget": ([_P, _P], _I),
    "ns_set_scheme": ([_P, _I], _I),
    "ns_set_cfl": ([_P, _D], _I),
    "ns_set_hyperviscosity": ([_P, _D, _D], _I),
    "ns_get_time": ([_P, _PD, _PD], _I),
    "ns_state_to_phys_device": ([_P, _P], _I),
    "ns_set_forcing_phys_device": ([_P, _P], _I),
    "ns_cnn_init": ([ctypes.POINTER(_P), _I, _I, _I, ctypes.c_ulonglong], _I),
    "ns_cnn_num_params": ([_P], _I),
    "ns_cnn_get_params": ([_P, _P], _I),
    "ns_cnn_set_params": ([_P, _P], _I),
    "ns_cnn_forward": ([_P, _P, _P, _I, _P], _I),
    "ns_cnn_gradients": ([_P, _P, _P, _I, _P, ctypes.POINTER(ctypes.c_float)], _I),
    "ns_cnn_train_step": ([_P, _P, _P, _I, ctypes.c_float, ctypes.POINTER(ctypes.c_float), _P], _I),
    "ns_cnn_destroy": ([_P], None),
    "ns_cnn_last_error": ([_P], ctypes.c_char_p),
    "ns_f64_to_f32": ([_P, _P, _LL, _D, _P], _I),
    "ns_f32_axpy_f64": ([_P, _P, _P, _LL, _D, _P], _I),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with __graft_entry__.build() "
                          "(the CUDA library is the only implementation)")
    lib = ctypes.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = load()


class NSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, state=None):
    if rc != NS_OK:
        msg = lib.ns_last_error(state)
        raise NSError(rc, msg.decode() if msg else "")


# ---------------------------------------------------- C-named functions ---
def ns_sizes(dim: int, n: int, precision: int):
    g = ns_grid(dim, n, precision)
    kc, c, h, nb = _I(), _I(), _I(), _I()
    sd, pd = _LL(), _LL()
    _check(lib.ns_sizes(ctypes.byref(g), ctypes.byref(kc), ctypes.byref(c), ctypes.byref(h), ctypes.byref(sd),
                        ctypes.byref(pd), ctypes.byref(nb)))
    return dict(kc=kc.value, c=c.value, h=h.value, state_doubles=sd.value, phys_doubles=pd.value, nbins=nb.value)


def ns_init(dim: int, n: int, precision: int, nu: float, dt: float, forcing_phys=None):
    g = ns_grid(dim, n, precision)
    out = _P()
    f = None if forcing_phys is None else np.ascontiguousarray(forcing_phys, dtype=np.float64)
    _check(lib.ns_init(ctypes.byref(out), ctypes.byref(g), float(nu), float(dt), None if f is None else _ptr(f)))
    return out


def ns_destroy(state) -> None:
    lib.ns_destroy(state)


def ns_step(state, nsteps: int) -> None:
    _check(lib.ns_step(state, int(nsteps)), state)


def ns_sync(state) -> None:
    _check(lib.ns_sync(state), state)


def fp32_fma_peak(device: int = 0) -> float:
    """Measured FP32 FMA rate of the device in TFLOP/s (ns_fp32_fma_peak)."""
    t = ctypes.c_double()
    _check(lib.ns_fp32_fma_peak(int(device), ctypes.byref(t)))
    return t.value


def ns_set_stream(state, stream_handle: int | None) -> None:
    _check(lib.ns_set_stream(state, ctypes.c_void_p(stream_handle) if stream_handle else None), state)


# ------------------------------------------------------------- wrapper ---
class Solver:
    """One solver state: ``Solver(dim, n, precision, nu, dt, forcing_phys=None)``.

    Arrays in and out follow the canonical layouts of include/ns.h: physical
    float64 ``(3, N, N, N)`` / ``(N, N)``; spectral complex128 ``(3, c, c, h)`` /
    ``(c, h)``.
    """

    def __init__(self, dim: int, n: int, precision: int = NS_FP32, nu: float = 0.0, dt: float = 1e-3,
                 forcing_phys=None):
        self.dim, self.n, self.precision = dim, n, precision
        self.sizes = ns_sizes(dim, n, precision)
        kc, c, h = self.sizes["kc"], self.sizes["c"], self.sizes["h"]
        self.spec_shape = (3, c, c, h) if dim == 3 else (c, h)
        self.phys_shape = (3, n, n, n) if dim == 3 else (n, n)
        if forcing_phys is not None:
            forcing_phys = np.ascontiguousarray(forcing_phys, dtype=np.float64).reshape(self.phys_shape)
        self.state = ns_init(dim, n, precision, nu, dt, forcing_phys)

    def close(self):
        if getattr(self, "state", None):
            ns_destroy(self.state)
            self.state = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_state(self, phys: np.ndarray) -> None:
        p = np.ascontiguousarray(phys, dtype=np.float64).reshape(self.phys_shape)
        _check(lib.ns_set_state(self.state, _ptr(p)), self.state)

    def get_state(self) -> np.ndarray:
        out = np.empty(self.phys_shape, np.float64)
        _check(lib.ns_get_state(self.state, _ptr(out)), self.state)
        return out

    def set_state_spectral(self, spec: np.ndarray) -> None:
        s = np.ascontiguousarray(spec, dtype=np.complex128).reshape(self.spec_shape)
        _check(lib.ns_set_state_spectral(self.state, _ptr(s)), self.state)

    def set_state_spectral_ptr(self, host_ptr: int) -> None:
        """Set from a raw host pointer (e.g. pinned memory) in the canonical layout."""
        _check(lib.ns_set_state_spectral(self.state, ctypes.c_void_p(host_ptr)), self.state)

    def get_state_spectral(self) -> np.ndarray:
        out = np.empty(self.spec_shape, np.complex128)
        _check(lib.ns_get_state_spectral(self.state, _ptr(out)), self.state)
        return out

    def get_state_spectral_ptr(self, host_ptr: int) -> None:
        _check(lib.ns_get_state_spectral(self.state, ctypes.c_void_p(host_ptr)), self.state)

    def step(self, nsteps: int) -> None:
        ns_step(self.state, nsteps)

    def sync(self) -> None:
        ns_sync(self.state)

    def eval_rhs(self) -> np.ndarray:
        out = np.empty(self.spec_shape, np.complex128)
        _check(lib.ns_eval_rhs(self.state, _ptr(out)), self.state)
        return out

    def diagnostics(self):
        e, o = _D(), _D()
        _check(lib.ns_diagnostics(self.state, ctypes.byref(e), ctypes.byref(o)), self.state)
        return e.value, o.value

    def set_scheme(self, order: int) -> None:
        """Lawson IF-RK of order 4 (default) or 2 (midpoint)."""
        _check(lib.ns_set_scheme(self.state, int(order)), self.state)

    def set_cfl(self, cfl: float) -> None:
        """CFL-adaptive dt (capped by the initial dt); 0 = constant dt."""
        _check(lib.ns_set_cfl(self.state, float(cfl)), self.state)

    def set_hyperviscosity(self, nu4: float, nu8: float = 0.0) -> None:
        """Add -(nu4 |k|^4 + nu8 |k|^8) to the linear operator (0, 0 removes it)."""
        _check(lib.ns_set_hyperviscosity(self.state, float(nu4), float(nu8)), self.state)

    def time(self):
        """(simulated time, dt of the last step)."""
        t, dt = _D(), _D()
        _check(lib.ns_get_time(self.state, ctypes.byref(t), ctypes.byref(dt)), self.state)
        return t.value, dt.value

    def budget(self):
        """(P_E, D_E, P_Z, D_Z): forcing power and dissipation of energy and enstrophy."""
        out = np.zeros(4, np.float64)
        _check(lib.ns_budget(self.state, _ptr(out)), self.state)
        return tuple(float(v) for v in out)

    def energy_spectrum(self) -> np.ndarray:
        nb = self.sizes["nbins"]
        out = np.zeros(nb, np.float64)
        cap = _I(nb)
        _check(lib.ns_energy_spectrum(self.state, _ptr(out), ctypes.byref(cap)), self.state)
        return out[: cap.value]

    def set_stream(self, stream_handle: int | None) -> None:
        ns_set_stream(self.state, stream_handle)

    def profile_step(self, nsteps: int):
        k = lib.ns_num_kernels()
        ms = np.zeros(k, np.float64)
        cnt = np.zeros(k, np.int32)
        _check(lib.ns_profile_step(self.state, int(nsteps), _ptr(ms), _ptr(cnt), k), self.state)
        names = [lib.ns_kernel_name(i).decode() for i in range(k)]
        return {names[i]: (float(ms[i]), int(cnt[i]), int(lib.ns_kernel_bytes(self.state, i))) for i in range(k)}

    def device_bytes(self) -> int:
        return int(lib.ns_device_bytes(self.state))


def _echeck(rc: int, ens=None):
    if rc != NS_OK:
        msg = lib.ns_ensemble_last_error(ens)
        raise NSError(rc, msg.decode() if msg else "")


class Ensemble:
    """Independent 2D runs of uneven sizes advanced together:
    ``Ensemble(sizes, precision, nu, dt, autotune=True)``.  Member states use
    the canonical 2D spectral layout ``(c, h)`` of their own grid."""

    def __init__(self, sizes, precision: int = NS_FP32, nu: float = 0.0, dt: float = 1e-3, autotune: bool = True):
        self.sizes = [int(n) for n in sizes]
        self.shapes = []
        for n in self.sizes:
            z = ns_sizes(2, n, precision)
            self.shapes.append((z["c"], z["h"]))
        arr = np.ascontiguousarray(self.sizes, dtype=np.int32)
        out = _P()
        _echeck(lib.ns_ensemble_init(ctypes.byref(out), len(self.sizes), _ptr(arr), precision, float(nu), float(dt),
                                     1 if autotune else 0))
        self.ens = out

    def close(self):
        if getattr(self, "ens", None):
            lib.ns_ensemble_destroy(self.ens)
            self.ens = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def schedule(self):
        a, b, c = _I(), _I(), _I()
        _echeck(lib.ns_ensemble_schedule(self.ens, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), self.ens)
        return a.value, b.value, c.value

    def set_schedule(self, x_blocks: int, y_blocks: int, order: int) -> None:
        _echeck(lib.ns_ensemble_set_schedule(self.ens, x_blocks, y_blocks, order), self.ens)

    def tiles(self):
        """(y-pass block threads, x-pass warps per block) of the schedule."""
        a, b = _I(), _I()
        _echeck(lib.ns_ensemble_tiles(self.ens, ctypes.byref(a), ctypes.byref(b)), self.ens)
        return a.value, b.value

    def set_tiles(self, y_threads: int, x_warps: int) -> None:
        _echeck(lib.ns_ensemble_set_tiles(self.ens, int(y_threads), int(x_warps)), self.ens)

    def fused(self):
        """(blocks per SM of the one-launch-per-stage form, 0 = two launches; the most allowed)."""
        a, b = _I(), _I()
        _echeck(lib.ns_ensemble_fused(self.ens, ctypes.byref(a), ctypes.byref(b)), self.ens)
        return a.value, b.value

    def set_fused(self, blocks_per_sm: int) -> None:
        _echeck(lib.ns_ensemble_set_fused(self.ens, int(blocks_per_sm)), self.ens)

    def set_state_spectral(self, member: int, spec) -> None:
        s = np.ascontiguousarray(spec, dtype=np.complex128).reshape(self.shapes[member])
        _echeck(lib.ns_ensemble_set_state_spectral(self.ens, member, _ptr(s)), self.ens)

    def get_state_spectral(self, member: int):
        out = np.empty(self.shapes[member], np.complex128)
        _echeck(lib.ns_ensemble_get_state_spectral(self.ens, member, _ptr(out)), self.ens)
        return out

    def step(self, nsteps: int) -> None:
        _echeck(lib.ns_ensemble_step(self.ens, int(nsteps)), self.ens)

    def sync(self) -> None:
        _echeck(lib.ns_ensemble_sync(self.ens), self.ens)

    def set_stream(self, stream_handle) -> None:
        _echeck(lib.ns_ensemble_set_stream(self.ens, ctypes.c_void_p(stream_handle) if stream_handle else None),
                self.ens)

    def diagnostics(self):
        e = np.zeros(len(self.sizes))
        o = np.zeros(len(self.sizes))
        _echeck(lib.ns_ensemble_diagnostics(self.ens, _ptr(e), _ptr(o)), self.ens)
        return e, o


# ------------------------------------------------------ learned closure ---
def _ccheck(rc: int, net=None):
    if rc != NS_OK:
        msg = lib.ns_cnn_last_error(net)
        raise NSError(rc, msg.decode() if msg else "")


class CNN:
    """The closure network of include/ns.h (4 periodic 3x3 convolutions,
    1 -> 32 -> 32 -> 32 -> 1 channels, GELU, BF16 storage, FP32 accumulation).

    ``forward``/``train_step`` take device pointers (ints, e.g. from
    ``torch.Tensor.data_ptr()``) to FP32 ``[batch][height][width]`` arrays.
    """

    def __init__(self, height: int, width: int, max_batch: int, seed: int = 0):
        self.height, self.width, self.max_batch = height, width, max_batch
        out = ctypes.c_void_p()
        _ccheck(lib.ns_cnn_init(ctypes.byref(out), height, width, max_batch, ctypes.c_ulonglong(seed)))
        self.net = out
        self.num_params = int(lib.ns_cnn_num_params(self.net))

    def close(self):
        if getattr(self, "net", None):
            lib.ns_cnn_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def get_params(self) -> np.ndarray:
        out = np.empty(self.num_params, np.float32)
        _ccheck(lib.ns_cnn_get_params(self.net, _ptr(out)), self.net)
        return out

    def set_params(self, p: np.ndarray) -> None:
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != self.num_params:
            raise ValueError(f"expected {self.num_params} parameters, got {p.size}")
        _ccheck(lib.ns_cnn_set_params(self.net, _ptr(p)), self.net)

    def forward(self, x_dev: int, y_dev: int, batch: int, stream: int | None = None) -> None:
        _ccheck(lib.ns_cnn_forward(self.net, ctypes.c_void_p(x_dev), ctypes.c_void_p(y_dev), batch,
                                   ctypes.c_void_p(stream) if stream else None), self.net)

    def gradients(self, x_dev: int, t_dev: int, batch: int):
        g = np.empty(self.num_params, np.float32)
        loss = ctypes.c_float()
        _ccheck(lib.ns_cnn_gradients(self.net, ctypes.c_void_p(x_dev), ctypes.c_void_p(t_dev), batch, _ptr(g),
                                     ctypes.byref(loss)), self.net)
        return g, float(loss.value)

    def train_step(self, x_dev: int, t_dev: int, batch: int, lr: float, stream: int | None = None,
                   want_loss: bool = True):
        loss = ctypes.c_float()
        _ccheck(lib.ns_cnn_train_step(self.net, ctypes.c_void_p(x_dev), ctypes.c_void_p(t_dev), batch,
                                      ctypes.c_float(lr), ctypes.byref(loss) if want_loss else None,
                                      ctypes.c_void_p(stream) if stream else None), self.net)
        return float(loss.value) if want_loss else None


def f64_to_f32(src_dev: int, dst_dev: int, n: int, scale: float = 1.0, stream: int | None = None) -> None:
    _check(lib.ns_f64_to_f32(ctypes.c_void_p(src_dev), ctypes.c_void_p(dst_dev), n, scale,
                             ctypes.c_void_p(stream) if stream else None))


def f32_axpy_f64(src_dev: int, base_dev: int | None, dst_dev: int, n: int, scale: float = 1.0,
                 stream: int | None = None) -> None:
    _check(lib.ns_f32_axpy_f64(ctypes.c_void_p(src_dev), ctypes.c_void_p(base_dev) if base_dev else None,
                               ctypes.c_void_p(dst_dev), n, scale, ctypes.c_void_p(stream) if stream else None))
