"""Pins of the oracle's budget terms (forcing power and dissipation) against
the time derivative of the oracle's own, independently pinned, energy and
enstrophy along its Lawson RK4 trajectories: for the Galerkin system the
nonlinear term conserves energy (2D and 3D) and enstrophy (2D), so
dE/dt = P_E - D_E and, in 2D, dOmega/dt = P_Z - D_Z; in 3D the vortex
stretching vanishes on a Beltrami field, so dOmega/dt = P_Z - D_Z there."""
import numpy as np
import pytest

from paper_1807_01769_gb300 import inputs


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


def forcing(orc, dim, n, seed):
    if dim == 2:
        return orc.phys_to_state(2, n, inputs.kolmogorov_forcing_2d(n, amp=4.0, k=2)) + \
            5.0 * inputs.random_vorticity_2d(n, seed=seed, k0=3.0)
    return 5.0 * inputs.random_velocity_3d(n, seed=seed, k0=2.0)


def rate(orc, dim, n, nu, h, u, f, which):
    """One-sided second-order derivative of E (which = 0) or Omega (1) at t = 0."""
    v = [orc.diagnostics(dim, n, orc.step(dim, n, nu, h, k, u, forcing=f) if k else u)[which] for k in range(3)]
    return (-3 * v[0] + 4 * v[1] - v[2]) / (2 * h)


@pytest.mark.parametrize("dim,n", [(2, 32), (3, 16)])
def test_energy_rate_equals_power_minus_dissipation(orc, dim, n):
    nu, h = 0.02, 1e-4
    u = inputs.random_vorticity_2d(n, seed=3, k0=3.0) if dim == 2 else inputs.random_velocity_3d(n, seed=3, k0=2.0)
    f = forcing(orc, dim, n, 11)
    pe, de, _, _ = orc.budget(dim, n, nu, u, f)
    assert abs(pe) > 0.1 * de > 0
    assert abs(rate(orc, dim, n, nu, h, u, f, 0) - (pe - de)) < 1e-5 * (abs(pe) + de)


def test_enstrophy_rate_2d(orc):
    n, nu, h = 32, 0.02, 1e-4
    u = inputs.random_vorticity_2d(n, seed=5, k0=3.0)
    f = forcing(orc, 2, n, 12)
    _, _, pz, dz = orc.budget(2, n, nu, u, f)
    assert abs(rate(orc, 2, n, nu, h, u, f, 1) - (pz - dz)) < 1e-5 * (abs(pz) + dz)


def test_enstrophy_rate_3d_beltrami(orc):
    n, nu, h = 16, 0.02, 1e-4
    u = orc.phys_to_state(3, n, inputs.abc_flow(n, 1.0, 0.7, 0.4))
    f = forcing(orc, 3, n, 13)
    _, _, pz, dz = orc.budget(3, n, nu, u, f)
    assert abs(rate(orc, 3, n, nu, h, u, f, 1) - (pz - dz)) < 1e-5 * (abs(pz) + dz)


@pytest.mark.parametrize("dim,n", [(2, 32), (3, 16)])
def test_dissipation_is_twice_nu_enstrophy_and_no_forcing_no_power(orc, dim, n):
    nu = 0.003
    u = inputs.random_vorticity_2d(n, seed=6) if dim == 2 else inputs.random_velocity_3d(n, seed=6)
    pe, de, pz, dz = orc.budget(dim, n, nu, u)
    _, om = orc.diagnostics(dim, n, u)
    assert pe == 0.0 and pz == 0.0
    assert abs(de - 2 * nu * om) < 1e-12 * de
    assert dz > 0


@pytest.mark.parametrize("dim,n", [(2, 32), (3, 16)])
def test_energy_rate_with_hyperviscosity(orc, dim, n):
    nu, nu4, nu8, h = 0.01, 1e-3, 1e-7, 1e-4
    u = inputs.random_vorticity_2d(n, seed=3, k0=3.0) if dim == 2 else inputs.random_velocity_3d(n, seed=3, k0=2.0)
    f = forcing(orc, dim, n, 11)
    pe, de, _, _ = orc.budget(dim, n, nu, u, f, nu4=nu4, nu8=nu8)
    _, de0, _, _ = orc.budget(dim, n, nu, u, f)
    assert de > 1.2 * de0  # the hyper terms matter at these coefficients
    v = [orc.diagnostics(dim, n, orc.step(dim, n, nu, h, k, u, forcing=f, nu4=nu4, nu8=nu8) if k else u)[0]
         for k in range(3)]
    rate = (-3 * v[0] + 4 * v[1] - v[2]) / (2 * h)
    assert abs(rate - (pe - de)) < 1e-5 * (abs(pe) + de)
