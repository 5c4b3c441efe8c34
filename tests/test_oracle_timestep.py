"""Pins of the oracle's order-2 Lawson step, its physical velocity and its
CFL-adaptive stepping: closed-form solutions, the convergence order and the
CFL rule on a field whose maximum velocity is known."""
import numpy as np
import pytest

from paper_1807_01769_gb300 import inputs


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


@pytest.mark.parametrize("dim,n,dt", [(2, 32, 0.02), (3, 16, 0.04)])
def test_rk2_second_order(orc, dim, n, dt):
    nu, t_end = 0.005, 0.64
    u0 = inputs.random_vorticity_2d(n, seed=0, k0=3.0) if dim == 2 else inputs.random_velocity_3d(n, seed=4, k0=2.0)
    ref = orc.step(dim, n, nu, dt / 32, int(round(32 * t_end / dt)), u0)  # RK4 with a small step
    e1 = np.linalg.norm(orc.step(dim, n, nu, dt, int(round(t_end / dt)), u0, order=2) - ref)
    e2 = np.linalg.norm(orc.step(dim, n, nu, dt / 2, int(round(2 * t_end / dt)), u0, order=2) - ref)
    assert e1 > 1e-8
    assert 3.5 < e1 / e2 < 4.6


def test_rk2_exact_on_a_linear_decay(orc):
    # 2D Taylor-Green: the nonlinear term vanishes, the integrating factor is exact
    n, nu, dt, steps = 32, 0.05, 0.1, 10
    w0 = orc.phys_to_state(2, n, inputs.taylor_green_vorticity_2d(n))
    got = orc.step(2, n, nu, dt, steps, w0, order=2)
    np.testing.assert_allclose(got, w0 * np.exp(-2 * nu * dt * steps), atol=1e-14)


def test_rk2_forced_single_mode_local_error(orc):
    # a single Fourier mode has no nonlinear term in 2D: dw/dt = -nu k^2 w + f,
    # exact w(dt) = E w0 + f (1 - E) / (nu k^2); the midpoint rule on the
    # integrating-factor integral errs by O(dt^3) per step
    n, nu = 16, 0.3
    kc, c, h = inputs.truncation(n)
    w0 = np.zeros((c, h), np.complex128)
    f = np.zeros_like(w0)
    w0[1, 2], f[1, 2] = 0.7 - 0.2j, 1.5 + 0.4j  # (ky, kx) = (1, 2), |k|^2 = 5
    lam = 5 * nu
    errs = []
    for dt in (0.2, 0.1):
        got = orc.step(2, n, nu, dt, 1, w0, forcing=f, order=2)
        e = np.exp(-lam * dt)
        exact = e * w0[1, 2] + f[1, 2] * (1 - e) / lam
        assert np.count_nonzero(np.abs(got) > 1e-14) == 1
        errs.append(abs(got[1, 2] - exact))
    assert 7.0 < errs[0] / errs[1] < 9.0


def test_velocity_of_taylor_green(orc):
    n = 16
    x = inputs.grid_coords(n)
    y2, x2 = np.meshgrid(x, x, indexing="ij")
    u = orc.velocity(2, n, orc.phys_to_state(2, n, inputs.taylor_green_vorticity_2d(n)))
    np.testing.assert_allclose(u[0], np.sin(x2) * np.cos(y2), atol=1e-13)
    np.testing.assert_allclose(u[1], -np.cos(x2) * np.sin(y2), atol=1e-13)
    s3 = orc.phys_to_state(3, n, inputs.taylor_green_3d(n))
    np.testing.assert_allclose(orc.velocity(3, n, s3), inputs.taylor_green_3d(n), atol=1e-13)


@pytest.mark.parametrize("order", [2, 4])
def test_cfl_rule(orc, order):
    # 3D Taylor-Green: max|u_x| = max|u_y| = 1 on grids with N divisible by 4,
    # u_z = 0 (ignored), so the first dt is cfl * 2 pi / N unless capped
    n, nu, cfl = 16, 0.01, 0.5
    s = orc.phys_to_state(3, n, inputs.taylor_green_3d(n))
    dx = 2 * np.pi / n
    _, dts = orc.step_cfl(3, n, nu, 1.0, cfl, 1, s, order=order)
    assert abs(dts[0] - cfl * dx) < 1e-14
    _, dts = orc.step_cfl(3, n, nu, 0.05, cfl, 1, s, order=order)
    assert dts[0] == 0.05
    # every step equals a plain step with the dt it reports
    u = inputs.random_vorticity_2d(32, seed=2, k0=3.0)
    got, dts = orc.step_cfl(2, 32, nu, 1.0, 0.4, 3, u, order=order)
    ref = u
    for dt in dts:
        vmax = np.abs(orc.velocity(2, 32, ref)).reshape(2, -1).max(axis=1)
        assert abs(dt - min(1.0, 0.4 * (2 * np.pi / 32) / vmax.max())) < 1e-15
        ref = orc.step(2, 32, nu, dt, 1, ref, order=order)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("order", [2, 4])
def test_hyperviscosity_exact_decay_of_a_single_2d_mode(orc, order):
    # one Fourier mode has no nonlinear term in 2D: w(t) = w0 exp(-(nu k^2 + nu4 k^4 + nu8 k^8) t)
    n, nu, nu4, nu8, dt, steps = 32, 0.01, 2e-4, 1e-8, 0.05, 8
    kc, c, h = inputs.truncation(n)
    w0 = np.zeros((c, h), np.complex128)
    w0[3, 4] = 0.8 + 0.3j  # (ky, kx) = (3, 4), |k|^2 = 25
    got = orc.step(2, n, nu, dt, steps, w0, order=order, nu4=nu4, nu8=nu8)
    rate = nu * 25 + nu4 * 25 ** 2 + nu8 * 25 ** 4
    np.testing.assert_allclose(got, w0 * np.exp(-rate * dt * steps), atol=1e-15)


def test_hyperviscosity_exact_decay_of_a_beltrami_field(orc):
    # ABC flow at |k| = 1: u x w = 0, each mode decays by exp(-(nu + nu4 + nu8) t)
    n, nu, nu4, nu8, dt, steps = 16, 0.02, 0.03, 0.01, 0.1, 5
    u0 = orc.phys_to_state(3, n, inputs.abc_flow(n))
    got = orc.step(3, n, nu, dt, steps, u0, nu4=nu4, nu8=nu8)
    np.testing.assert_allclose(got, u0 * np.exp(-(nu + nu4 + nu8) * dt * steps), atol=1e-14)


def test_zero_hyperviscosity_is_the_plain_step(orc):
    u0 = inputs.random_vorticity_2d(32, seed=4, k0=3.0)
    a = orc.step(2, 32, 0.01, 0.02, 5, u0)
    b = orc.step(2, 32, 0.01, 0.02, 5, u0, nu4=0.0, nu8=0.0)
    np.testing.assert_array_equal(a, b)
