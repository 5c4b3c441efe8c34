"""Pins of the oracle's nonlinear term, projection, integrating factor, RK4 and
diagnostics against the mathematics: direct Galerkin convolution sums on tiny
grids, closed-form decays of exact Navier-Stokes solutions, conservation laws
of the truncated Euler system, the RK4 convergence order and the energy budget."""
import numpy as np
import pytest

from paper_1807_01769_gb300 import inputs


# ----------------------------------------------------------------- helpers --
def full_cube(trunc, n):
    """Truncated half spectrum -> dict-like full cube of retained modes,
    indexed [k + kc] along every axis (kx last), using u(-k) = conj u(k)."""
    kc, c, h = inputs.truncation(n)
    idx = np.arange(-kc, kc + 1)
    it = np.where(idx >= 0, idx, idx + c)  # truncated index of wavenumber k
    if trunc.ndim == 2:  # 2D (ky, kx)
        out = np.zeros((c, c), np.complex128)
        for a, ky in enumerate(idx):
            for b, kx in enumerate(idx):
                if kx >= 0:
                    out[a, b] = trunc[it[a], kx]
                else:
                    out[a, b] = np.conj(trunc[it[c - 1 - a], -kx])
        return out
    out = np.zeros((3, c, c, c), np.complex128)
    for a, kz in enumerate(idx):
        for b, ky in enumerate(idx):
            for e, kx in enumerate(idx):
                if kx >= 0:
                    out[:, a, b, e] = trunc[:, it[a], it[b], kx]
                else:
                    out[:, a, b, e] = np.conj(trunc[:, it[c - 1 - a], it[c - 1 - b], -kx])
    return out


def galerkin_rhs_2d(w_trunc, n):
    """N(k) = -sum_{p+q=k} (u_hat(p) . i q) w_hat(q), all |k_i|,|p_i|,|q_i| <= kc."""
    kc, c, h = inputs.truncation(n)
    W = full_cube(w_trunc, n)
    k1 = np.arange(-kc, kc + 1)
    PY, PX = np.meshgrid(k1, k1, indexing="ij")
    p2 = PX ** 2 + PY ** 2
    psi = np.where(p2 > 0, W / np.where(p2 > 0, p2, 1), 0)
    ux, uy = 1j * PY * psi, -1j * PX * psi
    out = np.zeros((c, h), np.complex128)
    for iy in range(c):
        ky = iy if iy <= kc else iy - c
        for kx in range(h):
            qy, qx = ky - PY, kx - PX
            ok = (np.abs(qy) <= kc) & (np.abs(qx) <= kc)
            wq = np.where(ok, W[np.clip(qy + kc, 0, c - 1), np.clip(qx + kc, 0, c - 1)], 0)
            out[iy, kx] = -np.sum(ux * 1j * qx * wq + uy * 1j * qy * wq)
    out[0, 0] = 0
    return out


def galerkin_rhs_3d(u_trunc, n):
    """N(k) = P(k) sum_{p+q=k} u_hat(p) x (i q x u_hat(q)), projected."""
    kc, c, h = inputs.truncation(n)
    U = full_cube(u_trunc, n)
    k1 = np.arange(-kc, kc + 1)
    PZ, PY, PX = np.meshgrid(k1, k1, k1, indexing="ij")
    Wx = 1j * (PY * U[2] - PZ * U[1])
    Wy = 1j * (PZ * U[0] - PX * U[2])
    Wz = 1j * (PX * U[1] - PY * U[0])
    W = np.stack([Wx, Wy, Wz])
    out = np.zeros((3, c, c, h), np.complex128)
    for iz in range(c):
        kz = iz if iz <= kc else iz - c
        for iy in range(c):
            ky = iy if iy <= kc else iy - c
            for kx in range(h):
                qz, qy, qx = kz - PZ, ky - PY, kx - PX
                ok = (np.abs(qz) <= kc) & (np.abs(qy) <= kc) & (np.abs(qx) <= kc)
                sel = tuple(np.clip(q + kc, 0, c - 1) for q in (qz, qy, qx))
                wq = np.where(ok[None], W[(slice(None),) + sel], 0)
                nv = np.array([np.sum(U[1] * wq[2] - U[2] * wq[1]),
                               np.sum(U[2] * wq[0] - U[0] * wq[2]),
                               np.sum(U[0] * wq[1] - U[1] * wq[0])])
                kv = np.array([kx, ky, kz], float)
                k2 = kv @ kv
                if k2 > 0:
                    nv = nv - kv * (kv @ nv) / k2
                else:
                    nv[:] = 0
                out[:, iz, iy, kx] = nv
    return out


def kvec(n, dim):
    if dim == 2:
        kx, ky = inputs.wavenumbers(n, 2)
        return kx, ky
    return inputs.wavenumbers(n, 3)


# ------------------------------------------------------- nonlinear term ---
@pytest.mark.parametrize("n", [8, 16])
def test_rhs_2d_equals_galerkin_sum(orc, n):
    w = inputs.random_vorticity_2d(n, seed=5, k0=2.0)
    got = orc.rhs(2, n, w)
    ref = galerkin_rhs_2d(w, n)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_rhs_3d_equals_galerkin_sum(orc):
    n = 8
    u = inputs.random_velocity_3d(n, seed=9, k0=1.5)
    got = orc.rhs(3, n, u)
    ref = galerkin_rhs_3d(u, n)
    assert np.abs(ref).max() > 1e-3
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def _all_modes(n):
    kc, c, h = inputs.truncation(n)
    return [(kx, ky, kz) for kz in range(-kc, kc + 1) for ky in range(-kc, kc + 1) for kx in range(h)]


def _at(trunc, n, modes):
    kc, c, h = inputs.truncation(n)
    return np.array([[trunc[a, kz % c, ky % c, kx] for a in range(3)] for kx, ky, kz in modes])


def test_rhs_modes_equals_galerkin_sum(orc):
    # the oracle's sampled direct sum against the independent numpy sum
    n = 8
    u = inputs.random_velocity_3d(n, seed=9, k0=1.5)
    modes = _all_modes(n)
    got = orc.rhs_modes(n, u, modes)
    ref = _at(galerkin_rhs_3d(u, n), n, modes)
    assert np.abs(ref).max() > 1e-3
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_rhs_modes_equals_fft_rhs_with_forcing_and_non_hermitian_plane(orc):
    # two algorithms for one definition: the direct triad sum and the
    # pseudo-spectral product; the kx = 0 plane is deliberately not Hermitian
    # (both take its Hermitian part, the real part of the inverse transform)
    n = 16
    rng = np.random.default_rng(4)
    shape = orc.state_shape(3, n)
    u = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    f = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    modes = _all_modes(n)
    got = orc.rhs_modes(n, u, modes, f)
    ref = _at(orc.rhs(3, n, u, f), n, modes)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_rhs_modes_single_triad_closed_form(orc):
    # u holds two modes p and q (with their conjugates): at k = p + q only the
    # triads (p, q) and (q, p) contribute, N(k) = P(k)[u_p x (i q x u_q) + u_q x (i p x u_p)]
    n = 16
    p, q = np.array([1, 2, 0]), np.array([2, -1, 1])
    up, uq = np.array([0.3 + 0.1j, -0.2j, 0.5]), np.array([0.1, 0.4 - 0.3j, -0.25j])
    kc, c, h = inputs.truncation(n)
    u = np.zeros(orc.state_shape(3, n), np.complex128)
    u[:, p[2] % c, p[1] % c, p[0]] = up
    u[:, q[2] % c, q[1] % c, q[0]] = uq
    k = p + q
    nv = np.cross(up, np.cross(1j * q, uq)) + np.cross(uq, np.cross(1j * p, up))
    nv = nv - k * (k @ nv) / (k @ k)
    got = orc.rhs_modes(n, u, [tuple(int(x) for x in k)])[0]
    assert np.abs(got - nv).max() < 1e-15
    with pytest.raises(ValueError):
        orc.rhs_modes(n, u, [(-1, 0, 0)])  # kx must be in 0..kc


def test_rhs_3d_divergence_free(orc):
    n = 16
    u = inputs.random_velocity_3d(n, seed=2, k0=3.0)
    r = orc.rhs(3, n, u)
    kx, ky, kz = kvec(n, 3)
    div = kx * r[0] + ky * r[1] + kz * r[2]
    assert np.abs(div).max() <= 1e-14 * np.abs(r).max() * n


def test_projection_removes_gradients(orc):
    n = 16
    x = inputs.grid_coords(n)
    z3, y3, x3 = np.meshgrid(x, x, x, indexing="ij")
    phi_grad = np.stack([np.cos(x3 + 2 * y3), 2 * np.cos(x3 + 2 * y3), 3 * np.cos(3 * z3)])  # grad of a scalar
    s = orc.phys_to_state(3, n, phi_grad)
    assert np.abs(s).max() < 1e-15


def test_rhs_forcing_enters_linearly(orc):
    n = 16
    w = inputs.random_vorticity_2d(n, seed=1)
    f = orc.phys_to_state(2, n, inputs.kolmogorov_forcing_2d(n))
    assert np.abs(orc.rhs(2, n, w, f) - orc.rhs(2, n, w) - f).max() < 1e-14


# -------------------------------------------------- closed-form decays ---
def test_taylor_green_2d_exact_decay(orc):
    n, nu, dt, steps = 32, 0.05, 0.01, 20
    w0 = orc.phys_to_state(2, n, inputs.taylor_green_vorticity_2d(n))
    assert np.abs(orc.rhs(2, n, w0)).max() < 1e-14  # u . grad w vanishes
    w = orc.step(2, n, nu, dt, steps, w0)
    # |k|^2 = 2: omega(t) = omega(0) exp(-2 nu t), exactly with the integrating factor
    assert np.abs(w - w0 * np.exp(-2 * nu * dt * steps)).max() < 1e-14


def test_abc_flow_exact_decay(orc):
    n, nu, dt, steps = 16, 0.1, 0.02, 10
    u0 = orc.phys_to_state(3, n, inputs.abc_flow(n))
    assert np.abs(orc.rhs(3, n, u0)).max() < 1e-14  # Beltrami: u x omega = 0
    u = orc.step(3, n, nu, dt, steps, u0)
    assert np.abs(u - u0 * np.exp(-nu * dt * steps)).max() < 1e-14


def test_shear_flow_exact_decay(orc):
    n, k, nu, dt, steps = 16, 3, 0.02, 0.01, 10
    u0 = orc.phys_to_state(3, n, inputs.shear_flow(n, k))
    assert np.abs(orc.rhs(3, n, u0)).max() < 1e-13  # u x omega is a gradient
    u = orc.step(3, n, nu, dt, steps, u0)
    assert np.abs(u - u0 * np.exp(-nu * k * k * dt * steps)).max() < 1e-14


def test_taylor_green_3d_initial_invariants(orc):
    n, nu, dt = 32, 1.0 / 1600, 2e-3
    u0 = orc.phys_to_state(3, n, inputs.taylor_green_3d(n))
    e0, om0 = orc.diagnostics(3, n, u0)
    assert abs(e0 - 1 / 8) < 1e-15 and abs(om0 - 3 / 8) < 1e-14
    u1 = orc.step(3, n, nu, dt, 1, u0)
    e1, _ = orc.diagnostics(3, n, u1)
    assert abs((e1 - e0) / dt - (-0.75 * nu)) < 1e-3 * 0.75 * nu + 1e-12


# ---------------------------------------------- invariants and RK4 order ---
def drift(orc, dim, n, u0, dt, t_end):
    u = orc.step(dim, n, 0.0, dt, int(round(t_end / dt)), u0)
    e0, o0 = orc.diagnostics(dim, n, u0)
    e1, o1 = orc.diagnostics(dim, n, u)
    if dim == 2:
        return abs(e1 - e0) / e0, abs(o1 - o0) / o0
    return abs(e1 - e0) / e0, abs(helicity(n, u) - helicity(n, u0))


def helicity(n, u):
    kx, ky, kz = kvec(n, 3)
    wx = 1j * (ky * u[2] - kz * u[1])
    wy = 1j * (kz * u[0] - kx * u[2])
    wz = 1j * (kx * u[1] - ky * u[0])
    w = np.where(kx == 0, 1.0, 2.0)
    return np.sum(w * np.real(np.conj(u[0]) * wx + np.conj(u[1]) * wy + np.conj(u[2]) * wz))


def test_invariants_conserved_at_zero_viscosity(orc):
    # the truncated Euler system conserves E and Omega (2D), E and helicity
    # (3D); RK4 leaves a drift that shrinks at least 2^4 times when dt halves
    n = 32
    w0 = inputs.random_vorticity_2d(n, seed=0, k0=3.0)
    d1 = drift(orc, 2, n, w0, 0.02, 0.8)
    d2 = drift(orc, 2, n, w0, 0.01, 0.8)
    for a, b in zip(d1, d2):
        assert a < 1e-5 and a / b > 14.0
    u0 = inputs.random_velocity_3d(16, seed=4, k0=2.0)
    d1 = drift(orc, 3, 16, u0, 0.04, 0.8)
    d2 = drift(orc, 3, 16, u0, 0.02, 0.8)
    for a, b in zip(d1, d2):
        assert a < 1e-4 and a / b > 14.0


@pytest.mark.parametrize("dim,n,dt", [(2, 32, 0.02), (3, 16, 0.04)])
def test_rk4_fourth_order(orc, dim, n, dt):
    # global error of the state after a fixed time scales as dt^4: halving dt
    # divides it by ~16 (reference: the same scheme with dt/16)
    nu, t_end = 0.005, 0.64
    u0 = inputs.random_vorticity_2d(n, seed=0, k0=3.0) if dim == 2 else inputs.random_velocity_3d(n, seed=4, k0=2.0)
    ref = orc.step(dim, n, nu, dt / 16, int(round(16 * t_end / dt)), u0)
    e1 = np.linalg.norm(orc.step(dim, n, nu, dt, int(round(t_end / dt)), u0) - ref)
    e2 = np.linalg.norm(orc.step(dim, n, nu, dt / 2, int(round(2 * t_end / dt)), u0) - ref)
    assert e1 > 1e-12
    assert 13.0 < e1 / e2 < 19.0


@pytest.mark.parametrize("dim,n", [(2, 32), (3, 16)])
def test_energy_budget(orc, dim, n):
    nu, dt = 0.01, 1e-3
    u = inputs.random_vorticity_2d(n, seed=3, k0=3.0) if dim == 2 else inputs.random_velocity_3d(n, seed=3, k0=2.0)
    um = orc.step(dim, n, nu, dt, 5, u)
    u0 = orc.step(dim, n, nu, dt, 1, um)
    up = orc.step(dim, n, nu, dt, 1, u0)
    em, _ = orc.diagnostics(dim, n, um)
    ep, _ = orc.diagnostics(dim, n, up)
    _, om = orc.diagnostics(dim, n, u0)
    dedt = (ep - em) / (2 * dt)
    assert abs(dedt + 2 * nu * om) < 1e-4 * abs(2 * nu * om)


# ------------------------------------------------------------ diagnostics ---
@pytest.mark.parametrize("dim,n", [(2, 32), (3, 16)])
def test_spectrum_sums_to_energy_and_parseval(orc, dim, n):
    u = inputs.random_vorticity_2d(n, seed=8) if dim == 2 else inputs.random_velocity_3d(n, seed=8)
    e, om = orc.diagnostics(dim, n, u)
    spec = orc.spectrum(dim, n, u)
    assert spec.size == int(np.floor(np.sqrt(dim) * ((n - 1) // 3) + 0.5)) + 1
    assert np.isclose(spec.sum(), e, rtol=1e-13)
    phys = orc.state_to_phys(dim, n, u)
    if dim == 3:
        assert np.isclose(0.5 * (phys ** 2).sum(0).mean(), e, rtol=1e-12)
    else:
        assert np.isclose(0.5 * (phys ** 2).mean(), om, rtol=1e-12)


def test_spectrum_single_shell(orc):
    n = 16
    x = inputs.grid_coords(n)
    z3, y3, x3 = np.meshgrid(x, x, x, indexing="ij")
    # |k| = sqrt(9+16) = 5 exactly: all energy in shell 5
    u = np.stack([np.zeros_like(x3), np.zeros_like(x3), np.cos(3 * x3 + 4 * y3)])
    s = orc.phys_to_state(3, n, u)
    spec = orc.spectrum(3, n, s)
    assert np.isclose(spec[5], 0.25, rtol=1e-14) and abs(spec.sum() - spec[5]) < 1e-16


# ------------------------------------------------------ synthetic inputs ---
def test_random_inputs_are_hermitian_solenoidal_and_normalised(orc):
    n = 32
    u = inputs.random_velocity_3d(n, seed=1)
    kc, c, h = inputs.truncation(n)
    for iz in range(c):
        for iy in range(c):
            jz, jy = (c - iz) % c, (c - iy) % c
            assert np.allclose(u[:, iz, iy, 0], np.conj(u[:, jz, jy, 0]), atol=0)
    kx, ky, kz = kvec(n, 3)
    assert np.abs(kx * u[0] + ky * u[1] + kz * u[2]).max() < 1e-15
    assert np.isclose(orc.diagnostics(3, n, u)[0], 0.5, rtol=1e-13)
    w = inputs.random_vorticity_2d(n, seed=1)
    assert np.isclose(orc.diagnostics(2, n, w)[0], 0.5, rtol=1e-13)
    # real physical field round-trips through the oracle's transforms
    assert np.allclose(orc.phys_to_state(3, n, orc.state_to_phys(3, n, u)), u, atol=1e-15)


def test_random_inputs_share_modes_across_resolution():
    a = inputs.random_velocity_3d(32, seed=6)
    b = inputs.random_velocity_3d(64, seed=6)
    kc_a, c_a, h_a = inputs.truncation(32)
    kc_b, c_b, h_b = inputs.truncation(64)
    ia = np.arange(c_a)
    ka = np.where(ia <= kc_a, ia, ia - c_a)
    ib = np.where(ka >= 0, ka, ka + c_b)
    sub = b[:, ib][:, :, ib][..., :h_a]
    # equal up to the energy normalisation (the finer grid holds a little more
    # of the spectrum's tail): one real scale factor close to 1
    scale = np.vdot(a, sub) / np.vdot(a, a)
    assert abs(scale.imag) < 1e-14 and abs(scale.real - 1) < 1e-4
    assert np.abs(sub - scale.real * a).max() < 1e-15
