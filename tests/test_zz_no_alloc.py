"""ns_diagnostics_noalloc, the diagnostics entry point for host code that
cannot allocate device memory (an allocator hook, a process whose device
memory belongs to another framework): called through the C ABI on a spectrum
the caller holds on the device, twice in a row, it must give what the
allocating entry points ns_diagnostics / ns_energy_spectrum give for the same
state.  Its scratch is a static device array shared by every call; the first
call on a device loads the module that holds it, and the second call must
leave the device's free memory unchanged."""
import ctypes

import numpy as np
import pytest

from paper_1807_01769_gb300 import inputs

pytestmark = pytest.mark.gpu

REL = 1e-12  # same FP64 reduction, same summation order


def _call(ns, grid, dev_ptr, out_ptr, stream):
    return ns.lib.ns_diagnostics_noalloc(ctypes.byref(grid), ctypes.c_void_p(dev_ptr), ctypes.c_void_p(out_ptr),
                                         ctypes.c_void_p(stream) if stream else None)


@pytest.mark.parametrize("dim,n,prec", [(2, 128, 0), (3, 64, 1), (3, 256, 1), (2, 2048, 1)])
def test_noalloc_matches_allocating_entry_points(dim, n, prec):
    torch = pytest.importorskip("torch")
    from paper_1807_01769_gb300 import ns

    u0 = inputs.random_vorticity_2d(n, seed=11) if dim == 2 else inputs.random_velocity_3d(n, seed=11)
    with ns.Solver(dim, n, prec, nu=1e-3, dt=1e-3) as s:
        s.set_state_spectral(u0)
        s.step(2)
        e_ref, om_ref = s.diagnostics()
        spec_ref = s.energy_spectrum()
        u = s.get_state_spectral()
        nb = s.sizes["nbins"]
    ctype = np.complex128 if prec == ns.NS_FP64 else np.complex64
    dev = torch.from_numpy(np.ascontiguousarray(u.astype(ctype))).to("cuda")
    out = torch.full((nb + 2,), float("nan"), dtype=torch.float64, device="cuda")
    grid = ns.ns_grid(dim, n, prec)
    stream = torch.cuda.current_stream().cuda_stream
    for i in range(2):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert _call(ns, grid, dev.data_ptr(), out.data_ptr(), stream) == ns.NS_OK
        torch.cuda.synchronize()
        if i == 1:  # after the warm-up call: nothing is allocated on the device
            assert torch.cuda.mem_get_info()[0] == free0
        got = out.cpu().numpy()
        assert abs(got[0] - e_ref) <= REL * e_ref
        assert abs(got[1] - om_ref) <= REL * om_ref
        assert np.allclose(got[2:], spec_ref, rtol=REL, atol=1e-300)
        out.fill_(float("nan"))  # the next call must rewrite every output


def test_noalloc_rejects_what_it_cannot_hold():
    torch = pytest.importorskip("torch")
    from paper_1807_01769_gb300 import ns

    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    # 512^3 needs more partial sums than the static scratch holds: refused on
    # the host before any launch
    assert _call(ns, ns.ns_grid(3, 512, 1), p, p, 0) == ns.NS_EUNSUPPORTED
    assert _call(ns, ns.ns_grid(3, 100, 1), p, p, 0) == ns.NS_EINVAL
    assert ns.lib.ns_diagnostics_noalloc(ctypes.byref(ns.ns_grid(2, 64, 1)), None, ctypes.c_void_p(p), None) \
        == ns.NS_EINVAL
