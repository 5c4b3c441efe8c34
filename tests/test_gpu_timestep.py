"""GPU parity of the order-2 Lawson step, the CFL-adaptive stepping and the
budget diagnostics against the FP64 oracle (same tolerances as the RK4
parity: relative L2 over the spectrum 1e-11 FP64, 1e-5 FP32 after the steps;
the CFL time steps to 1e-12 FP64 and 5e-6 FP32, where the maxima of |u| are
taken in the state precision)."""
import numpy as np
import pytest

from paper_1807_01769_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1
TOL = {FP64: 1e-11, FP32: 1e-5}
TOL_DT = {FP64: 1e-12, FP32: 5e-6}


@pytest.fixture(scope="module")
def ns():
    from paper_1807_01769_gb300 import ns as mod

    return mod


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


def rel_l2(a, b):
    w = np.where(np.arange(b.shape[-1]) == 0, 1.0, 2.0)
    return float(np.sqrt(np.sum(w * np.abs(a - b) ** 2) / np.sum(w * np.abs(b) ** 2)))


def ic(dim, n, seed=0):
    if dim == 2:
        return inputs.random_vorticity_2d(n, seed=seed, k0=8.0, a=1.0, energy=0.5)
    return inputs.random_velocity_3d(n, seed=seed, k0=4.0, a=2.0, energy=0.5)


@pytest.mark.parametrize("dim,n,prec", [(2, 64, FP64), (2, 256, FP32), (3, 32, FP64), (3, 64, FP32)])
def test_rk2_matches_oracle(ns, orc, dim, n, prec):
    nu, dt, steps = 2e-3, 2e-3, 10
    u0 = ic(dim, n)
    ref = orc.step(dim, n, nu, dt, steps, u0, order=2)
    with ns.Solver(dim, n, prec, nu=nu, dt=dt) as s:
        s.set_scheme(2)
        s.set_state_spectral(u0)
        s.step(steps)
        got = s.get_state_spectral()
        t, dtl = s.time()
    assert rel_l2(got, ref) < TOL[prec]
    assert abs(t - steps * dt) < 1e-15 and dtl == dt


def test_scheme_switch_back_to_rk4(ns, orc):
    n, nu, dt = 64, 2e-3, 2e-3
    u0 = ic(2, n)
    ref = orc.step(2, n, nu, dt, 3, orc.step(2, n, nu, dt, 4, u0, order=2))
    with ns.Solver(2, n, FP64, nu=nu, dt=dt) as s:
        s.set_state_spectral(u0)
        s.set_scheme(2)
        s.step(4)
        s.set_scheme(4)
        s.step(3)
        got = s.get_state_spectral()
    assert rel_l2(got, ref) < TOL[FP64]


@pytest.mark.parametrize("dim,n,prec,order", [(2, 64, FP64, 4), (2, 128, FP32, 4), (2, 64, FP64, 2),
                                              (3, 32, FP64, 4), (3, 64, FP32, 4), (3, 32, FP32, 2)])
def test_cfl_stepping_matches_oracle(ns, orc, dim, n, prec, order):
    nu, dt_max, cfl, steps = 2e-3, 0.05, 0.6, 8
    u0 = 4.0 * ic(dim, n, seed=2)  # fast enough that the CFL rule, not dt_max, sets dt
    ref, dts = orc.step_cfl(dim, n, nu, dt_max, cfl, steps, u0, order=order)
    assert np.all(dts < dt_max)
    with ns.Solver(dim, n, prec, nu=nu, dt=dt_max) as s:
        s.set_scheme(order)
        s.set_state_spectral(u0)
        s.set_cfl(cfl)
        got_dts = []
        for _ in range(steps):
            s.step(1)
            got_dts.append(s.time()[1])
        t, _ = s.time()
        got = s.get_state_spectral()
    np.testing.assert_allclose(got_dts, dts, rtol=TOL_DT[prec], atol=0)
    assert abs(t - dts.sum()) <= TOL_DT[prec] * dts.sum()
    assert rel_l2(got, ref) < TOL[prec]


def test_cfl_off_returns_to_constant_dt(ns, orc):
    n, nu, dt0, cfl = 64, 2e-3, 4e-3, 0.3
    u0 = 4.0 * ic(2, n, seed=3)
    mid, dts = orc.step_cfl(2, n, nu, dt0, cfl, 5, u0)
    assert np.all(dts < dt0)
    ref = orc.step(2, n, nu, dt0, 4, mid)
    with ns.Solver(2, n, FP64, nu=nu, dt=dt0) as s:
        s.set_state_spectral(u0)
        s.set_cfl(cfl)
        s.step(5)
        t5, _ = s.time()
        s.set_cfl(0.0)
        s.step(4)
        got = s.get_state_spectral()
        t, dt = s.time()
    assert abs(t5 - dts.sum()) < 1e-13
    assert abs(t - (t5 + 4 * dt0)) < 1e-13 and dt == dt0
    assert rel_l2(got, ref) < TOL[FP64]


def test_bad_scheme_and_cfl_rejected(ns):
    with ns.Solver(2, 32, FP32, nu=1e-3, dt=1e-3) as s:
        for order in (1, 3, 5):
            with pytest.raises(ns.NSError) as ei:
                s.set_scheme(order)
            assert ei.value.code == ns.NS_EINVAL
        for c in (-0.1, float("nan"), float("inf")):
            with pytest.raises(ns.NSError) as ei:
                s.set_cfl(c)
            assert ei.value.code == ns.NS_EINVAL


@pytest.mark.parametrize("dim,n,prec", [(2, 128, FP64), (2, 256, FP32), (3, 32, FP64), (3, 64, FP32)])
def test_budget_matches_oracle(ns, orc, dim, n, prec):
    nu = 3e-3
    u = ic(dim, n, seed=5)
    if dim == 2:
        f_phys = inputs.kolmogorov_forcing_2d(n, amp=4.0, k=4)
    else:
        f_phys = orc.state_to_phys(3, n, ic(3, n, seed=6))
    f_spec = orc.phys_to_state(dim, n, f_phys)
    ref = orc.budget(dim, n, nu, u, f_spec)
    with ns.Solver(dim, n, prec, nu=nu, dt=1e-3, forcing_phys=f_phys) as s:
        s.set_state_spectral(u)
        got = s.budget()
    tol = 1e-11 if prec == FP64 else 1e-5
    for a, b in zip(got, ref):
        assert abs(a - b) <= tol * max(abs(b), 1e-3 * max(abs(r) for r in ref)), (got, ref)
    with ns.Solver(dim, n, prec, nu=nu, dt=1e-3) as s:  # no forcing: no injection
        s.set_state_spectral(u)
        pe, de, pz, dz = s.budget()
        e, om = s.diagnostics()
    assert pe == 0.0 and pz == 0.0
    assert abs(de - 2 * nu * om) < 1e-12 * de


def test_rk2_with_forcing_matches_oracle(ns, orc):
    n, nu, dt, steps = 128, 1e-3, 2e-3, 10
    u0 = ic(2, n, seed=7)
    f_phys = inputs.kolmogorov_forcing_2d(n)
    ref = orc.step(2, n, nu, dt, steps, u0, forcing=orc.phys_to_state(2, n, f_phys), order=2)
    for prec in (FP64, FP32):
        with ns.Solver(2, n, prec, nu=nu, dt=dt, forcing_phys=f_phys) as s:
            s.set_scheme(2)
            s.set_state_spectral(u0)
            s.step(steps)
            assert rel_l2(s.get_state_spectral(), ref) < TOL[prec]


@pytest.mark.parametrize("dim,n", [(2, 64), (3, 32)])
def test_cfl_on_a_zero_field_takes_the_initial_dt(ns, dim, n):
    dt0 = 3e-3
    with ns.Solver(dim, n, FP64, nu=1e-3, dt=dt0) as s:
        s.set_state_spectral(np.zeros_like(ic(dim, n)))
        s.set_cfl(0.5)
        s.step(4)
        t, dt = s.time()
        assert dt == dt0 and abs(t - 4 * dt0) < 1e-15
        assert not np.any(s.get_state_spectral())


def test_cfl_with_3d_forcing_matches_oracle(ns, orc):
    n, nu, dt_max, cfl, steps = 32, 2e-3, 0.05, 0.5, 6
    u0 = 4.0 * ic(3, n, seed=8)
    f_phys = orc.state_to_phys(3, n, ic(3, n, seed=9))
    ref, dts = orc.step_cfl(3, n, nu, dt_max, cfl, steps, u0, forcing=orc.phys_to_state(3, n, f_phys))
    with ns.Solver(3, n, FP64, nu=nu, dt=dt_max, forcing_phys=f_phys) as s:
        s.set_state_spectral(u0)
        s.set_cfl(cfl)
        s.step(steps)
        t, dt = s.time()
        got = s.get_state_spectral()
    assert abs(t - dts.sum()) < 1e-12 * dts.sum() and abs(dt - dts[-1]) < 1e-12 * dts[-1]
    assert rel_l2(got, ref) < TOL[FP64]


def test_budget_without_viscosity_has_no_dissipation(ns, orc):
    n = 64
    u = ic(2, n, seed=10)
    f_phys = inputs.kolmogorov_forcing_2d(n)
    with ns.Solver(2, n, FP64, nu=0.0, dt=1e-3, forcing_phys=f_phys) as s:
        s.set_state_spectral(u)
        pe, de, pz, dz = s.budget()
    ref = orc.budget(2, n, 0.0, u, orc.phys_to_state(2, n, f_phys))
    assert de == 0.0 and dz == 0.0
    assert abs(pe - ref[0]) < 1e-12 * abs(ref[0]) and abs(pz - ref[2]) < 1e-12 * abs(ref[2])


@pytest.mark.parametrize("dim,n,prec,order", [(2, 64, FP64, 4), (2, 128, FP32, 4), (2, 64, FP64, 2),
                                              (3, 32, FP64, 4), (3, 64, FP32, 4), (3, 32, FP32, 2)])
def test_hyperviscosity_matches_oracle(ns, orc, dim, n, prec, order):
    nu, dt, steps = 2e-3, 2e-3, 10
    nu4, nu8 = (2e-5, 1e-11) if dim == 2 else (1e-3, 1e-9)  # visible on each initial field
    u0 = ic(dim, n, seed=11)
    ref = orc.step(dim, n, nu, dt, steps, u0, order=order, nu4=nu4, nu8=nu8)
    plain = orc.step(dim, n, nu, dt, steps, u0, order=order)
    assert rel_l2(ref, plain) > 1e3 * TOL[FP32]  # the hyper terms are visible
    with ns.Solver(dim, n, prec, nu=nu, dt=dt) as s:
        s.set_scheme(order)
        s.set_hyperviscosity(nu4, nu8)
        s.set_state_spectral(u0)
        s.step(steps)
        got = s.get_state_spectral()
        s.set_hyperviscosity(0.0, 0.0)  # back to plain viscosity
        s.set_state_spectral(u0)
        s.step(steps)
        got_plain = s.get_state_spectral()
    assert rel_l2(got, ref) < TOL[prec]
    assert rel_l2(got_plain, plain) < TOL[prec]


def test_hyperviscosity_budget_and_exclusions(ns, orc):
    n, nu, nu4, nu8 = 64, 1e-3, 1e-5, 1e-12
    u = ic(2, n, seed=12)
    f_phys = inputs.kolmogorov_forcing_2d(n)
    ref = orc.budget(2, n, nu, u, orc.phys_to_state(2, n, f_phys), nu4=nu4, nu8=nu8)
    with ns.Solver(2, n, FP64, nu=nu, dt=1e-3, forcing_phys=f_phys) as s:
        s.set_state_spectral(u)
        s.set_hyperviscosity(nu4, nu8)
        got = s.budget()
        for a, b in zip(got, ref):
            assert abs(a - b) <= 1e-11 * max(abs(b), 1e-3 * max(abs(r) for r in ref))
        with pytest.raises(ns.NSError) as ei:
            s.set_cfl(0.5)
        assert ei.value.code == ns.NS_EUNSUPPORTED
        s.set_hyperviscosity(0.0, 0.0)
        s.set_cfl(0.5)
        with pytest.raises(ns.NSError) as ei:
            s.set_hyperviscosity(1e-5, 0.0)
        assert ei.value.code == ns.NS_EUNSUPPORTED
        for bad in ((-1e-5, 0.0), (0.0, float("nan"))):
            with pytest.raises(ns.NSError) as ei:
                s.set_hyperviscosity(*bad)
            assert ei.value.code == ns.NS_EINVAL
