"""The C-ABI library loads and exports every symbol include/ns.h declares;
host-side argument checks return error codes without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "ns.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ns_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def ns():
    from paper_1807_01769_gb300 import build

    build.build()
    from paper_1807_01769_gb300 import ns as mod

    return mod


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["ns_init", "ns_step", "ns_energy_spectrum", "ns_set_state", "ns_get_state", "ns_diagnostics",
                 "ns_destroy", "ns_last_error", "ns_set_stream"]:
        assert name in syms


def test_library_exports_every_declared_symbol(ns):
    lib = ctypes.CDLL(ns.LIB_PATH)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    assert set(declared_symbols()) == set(ns.SIGNATURES)


def test_sizes(ns):
    s = ns.ns_sizes(3, 512, ns.NS_FP32)
    assert (s["kc"], s["c"], s["h"], s["nbins"]) == (170, 341, 171, 295)
    assert s["state_doubles"] == 2 * 3 * 341 * 341 * 171
    s = ns.ns_sizes(2, 128, ns.NS_FP64)
    assert (s["kc"], s["c"], s["h"], s["nbins"]) == (42, 85, 43, 60)


def test_tensor_core_precision_grids(ns):
    # NS_FP32_TC: 3D grids with a tensor-core x pass (64 .. 512) share the FP32 sizes
    for n in (64, 128, 256, 512):
        assert ns.ns_sizes(3, n, ns.NS_FP32_TC) == ns.ns_sizes(3, n, ns.NS_FP32)


@pytest.mark.parametrize("dim,n,prec,code", [(4, 64, 1, -1), (3, 100, 1, -1), (3, 8, 1, -4), (3, 2048, 1, -4),
                                              (2, 4096, 1, -4), (2, 64, 7, -1), (2, 256, 2, -4), (3, 32, 2, -4),
                                              (3, 1024, 2, -4)])
def test_bad_grids_rejected(ns, dim, n, prec, code):
    with pytest.raises(ns.NSError) as ei:
        ns.ns_sizes(dim, n, prec)
    assert ei.value.code == code


@pytest.mark.parametrize("nu,dt", [(-1.0, 1e-3), (1e-3, 0.0), (1e-3, -1.0), (float("nan"), 1e-3)])
def test_bad_parameters_rejected_before_any_device_call(ns, nu, dt):
    with pytest.raises(ns.NSError) as ei:
        ns.ns_init(2, 64, ns.NS_FP32, nu, dt)
    assert ei.value.code == ns.NS_EINVAL


def test_null_state_calls_return_einval(ns):
    assert ns.lib.ns_step(None, 1) == ns.NS_EINVAL
    assert ns.lib.ns_sync(None) == ns.NS_EINVAL
    assert ns.lib.ns_set_state(None, None) == ns.NS_EINVAL
    assert ns.lib.ns_kernel_bytes(None, 0) == -1
    ns.lib.ns_destroy(None)
    assert ns.lib.ns_num_kernels() == 5
    assert [ns.lib.ns_kernel_name(i).decode() for i in range(5)] == ["inv1", "inv2", "xpass", "fwd2", "fwd1"]


def test_ensemble_argument_checks(ns):
    import numpy as np

    with pytest.raises(ns.NSError) as ei:
        ns.Ensemble([128, 1024], ns.NS_FP32, nu=1e-3, dt=1e-3)
    assert ei.value.code == ns.NS_EUNSUPPORTED
    with pytest.raises(ns.NSError) as ei:
        ns.Ensemble([128], ns.NS_FP32, nu=-1.0, dt=1e-3)
    assert ei.value.code == ns.NS_EINVAL
    out = ns.ctypes.c_void_p()
    sizes = np.array([128], np.int32)
    assert ns.lib.ns_ensemble_init(ns.ctypes.byref(out), 0, sizes.ctypes.data_as(ns.ctypes.c_void_p), 1, 1e-3, 1e-3,
                                   0) == ns.NS_EINVAL
    assert ns.lib.ns_ensemble_step(None, 1) == ns.NS_EINVAL


def test_ensemble_sizes_draw():
    from paper_1807_01769_gb300 import inputs

    s = inputs.ensemble_sizes(64)
    assert len(s) == 64 and set(s) <= {128, 256, 512}
    assert s == inputs.ensemble_sizes(64)


def test_new_entry_points_check_arguments_before_any_device_call(ns):
    L, E = ns.lib, ns.NS_EINVAL
    d = ns.ctypes.c_double()
    assert L.ns_set_scheme(None, 2) == E
    assert L.ns_set_cfl(None, 0.5) == E
    assert L.ns_set_hyperviscosity(None, 1e-5, 0.0) == E
    assert L.ns_get_time(None, ns.ctypes.byref(d), ns.ctypes.byref(d)) == E
    assert L.ns_budget(None, None) == E
    assert L.ns_state_to_phys_device(None, None) == E
    assert L.ns_set_forcing_phys_device(None, None) == E
    assert L.ns_f64_to_f32(None, None, 10, 1.0, None) == E
    assert L.ns_f32_axpy_f64(None, None, None, 10, 1.0, None) == E
    assert L.ns_cnn_num_params(None) == -1
    assert L.ns_cnn_get_params(None, None) == E
    assert L.ns_cnn_set_params(None, None) == E
    assert L.ns_cnn_forward(None, None, None, 1, None) == E
    f = ns.ctypes.c_float()
    assert L.ns_cnn_gradients(None, None, None, 1, None, ns.ctypes.byref(f)) == E
    assert L.ns_cnn_train_step(None, None, None, 1, 1e-3, None, None) == E
    L.ns_cnn_destroy(None)
    assert L.ns_fp32_fma_peak(0, None) == E


@pytest.mark.parametrize("h,w,b", [(48, 64, 1), (64, 100, 1), (32, 32, 1), (64, 64, 0)])
def test_cnn_rejects_bad_shapes_without_a_device(ns, h, w, b):
    out = ns.ctypes.c_void_p()
    assert ns.lib.ns_cnn_init(ns.ctypes.byref(out), h, w, b, 0) == ns.NS_EINVAL
    assert not out.value
    assert b"multiples of 64" in ns.lib.ns_cnn_last_error(None)
