"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds no arithmetic of the method itself (no FFT, no projection,
no nonlinear term, no time stepping): it only builds initial conditions and
forcing fields, either in closed form in physical space or directly as
spectral coefficients on the retained (2/3-rule) modes.

The paper runs its benchmarks on "initial value problems with random fields"
(Performance / 2D benchmarks) without saying how they are drawn.  The reading
used here: fixed amplitude per shell, uniform random phase.  Random numbers
come from a counter-based generator (splitmix64, Steele, Lea & Flood 2014)
keyed by the wavevector, not by an array index, so a field drawn on a 64^3
grid and on a 512^3 grid with the same seed agree on every mode they share.

Spectral layouts (complex128) are the truncated ones: 3D ``(3, c, c, h)`` =
(comp, kz, ky, kx) and 2D ``(c, h)`` = (ky, kx), ``kc = (N-1)//3``,
``c = 2 kc + 1``, ``h = kc + 1``; index ``i`` on a full axis holds ``k = i`` for
``i <= kc`` and ``k = i - c`` otherwise.
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 output function applied to counters ``x`` (uint64, wraps)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, kx, ky, kz, stream: int) -> np.ndarray:
    """Uniform [0, 1) numbers keyed by (seed, wavevector, stream)."""
    kx = np.asarray(kx, dtype=np.int64)
    ky = np.asarray(ky, dtype=np.int64)
    kz = np.asarray(kz, dtype=np.int64)
    key = (((kz + 4096) << 26) | ((ky + 4096) << 13) | (kx + 4096)).astype(np.uint64)
    with np.errstate(over="ignore"):
        ctr = (key * np.uint64(16) + np.uint64(stream)) ^ splitmix64(np.uint64(seed))
        r = splitmix64(splitmix64(ctr))
    return (r >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def truncation(n: int):
    """(kc, c, h) for N points per axis (2/3 rule kept per axis)."""
    kc = (n - 1) // 3
    return kc, 2 * kc + 1, kc + 1


def wavenumbers(n: int, dim: int):
    """Integer wavevector arrays on the truncated layout: (kx, ky[, kz])."""
    kc, c, h = truncation(n)
    i = np.arange(c)
    kfull = np.where(i <= kc, i, i - c)
    kxa = np.arange(h)
    if dim == 2:
        ky, kx = np.meshgrid(kfull, kxa, indexing="ij")
        return kx, ky
    kz, ky, kx = np.meshgrid(kfull, kfull, kxa, indexing="ij")
    return kx, ky, kz


def k4_gauss_spectrum(k, k0: float, a: float):
    """E(k) proportional to k^4 exp(-a (k/k0)^2)."""
    k = np.asarray(k, dtype=np.float64)
    return k ** 4 * np.exp(-a * (k / k0) ** 2)


def _canonical(kx, ky, kz):
    """Flip modes of the kx = 0 plane into one half so that k and -k share
    random numbers; returns (kx', ky', kz', flipped)."""
    flip = (kx == 0) & ((kz < 0) | ((kz == 0) & (ky < 0)))
    return kx, np.where(flip, -ky, ky), np.where(flip, -kz, kz), flip


def random_vorticity_2d(n: int, seed: int, k0: float = 8.0, a: float = 1.0, energy: float = 0.5) -> np.ndarray:
    """Truncated 2D vorticity spectrum with |omega_hat| ~ sqrt(k E(k)),
    E(k) ~ k^4 exp(-a (k/k0)^2), random phases, Hermitian on kx = 0, zero
    mean, scaled so that the mean kinetic energy equals ``energy``."""
    kx, ky = wavenumbers(n, 2)
    kz = np.zeros_like(kx)
    kxc, kyc, kzc, flip = _canonical(kx, ky, kz)
    k2 = (kx * kx + ky * ky).astype(np.float64)
    k = np.sqrt(k2)
    amp = np.sqrt(k * k4_gauss_spectrum(k, k0, a))
    phase = 2.0 * np.pi * uniform01(seed, kxc, kyc, kzc, 0)
    w = amp * np.exp(1j * phase)
    w = np.where(flip, np.conj(w), w)
    w[k2 == 0] = 0.0
    weight = np.where(kx == 0, 1.0, 2.0)
    e = np.sum(weight * 0.5 * np.abs(w) ** 2 / np.where(k2 > 0, k2, 1.0))
    if e > 0:
        w *= np.sqrt(energy / e)
    return np.ascontiguousarray(w.astype(np.complex128))


def _solenoidal_modes(kx, ky, kz, seed: int, amp_of_k):
    """Random solenoidal coefficients on the given modes (arrays of equal
    shape): each mode is amp(|k|) (cos a e^{i p1} e1 + sin a e^{i p2} e2) with
    e1, e2 an orthonormal pair perpendicular to the canonical k; modes of the
    kx = 0 plane take the conjugate of their canonical partner, so that plane
    is Hermitian; the k = 0 mode is zero.  Returns (3, ...) complex128."""
    kxc, kyc, kzc, flip = _canonical(kx, ky, kz)
    kv = np.stack([kxc, kyc, kzc]).astype(np.float64)
    k2 = (kv ** 2).sum(0)
    k = np.sqrt(k2)
    kperp = np.sqrt(kv[0] ** 2 + kv[1] ** 2)
    on_axis = kperp == 0
    safe = np.where(on_axis, 1.0, kperp)
    e1 = np.stack([np.where(on_axis, 1.0, kv[1] / safe),
                   np.where(on_axis, 0.0, -kv[0] / safe),
                   np.zeros_like(k)])
    ksafe = np.where(k == 0, 1.0, k)
    e2 = np.stack([kv[1] * e1[2] - kv[2] * e1[1],
                   kv[2] * e1[0] - kv[0] * e1[2],
                   kv[0] * e1[1] - kv[1] * e1[0]]) / ksafe
    e2 = np.where(on_axis[None], np.stack([np.zeros_like(k), np.ones_like(k), np.zeros_like(k)]), e2)
    amp = amp_of_k(k, ksafe)
    p1 = 2.0 * np.pi * uniform01(seed, kxc, kyc, kzc, 1)
    p2 = 2.0 * np.pi * uniform01(seed, kxc, kyc, kzc, 2)
    al = 2.0 * np.pi * uniform01(seed, kxc, kyc, kzc, 3)
    u = amp * (np.cos(al) * np.exp(1j * p1) * e1 + np.sin(al) * np.exp(1j * p2) * e2)
    u = np.where(flip[None], np.conj(u), u)
    u[:, k2 == 0] = 0.0
    return u


def random_velocity_3d(n: int, seed: int, k0: float = 4.0, a: float = 2.0, energy: float = 0.5) -> np.ndarray:
    """Truncated 3D solenoidal velocity spectrum, |u_hat| ~ sqrt(E(k))/k with
    E(k) ~ k^4 exp(-a (k/k0)^2).  Each mode is a random combination of two unit
    vectors perpendicular to k with random phases, so k . u_hat = 0 holds by
    construction; Hermitian on kx = 0; zero mean; mean energy = ``energy``."""
    kx, ky, kz = wavenumbers(n, 3)
    u = _solenoidal_modes(kx, ky, kz, seed, lambda k, ksafe: np.sqrt(k4_gauss_spectrum(k, k0, a)) / ksafe)
    weight = np.where(kx == 0, 1.0, 2.0)
    e = np.sum(weight * 0.5 * (np.abs(u) ** 2).sum(0))
    if e > 0:
        u *= np.sqrt(energy / e)
    return np.ascontiguousarray(u.astype(np.complex128))


def random_velocity_3d_flat(n: int, seed: int, energy: float = 0.5, planes: int = 16) -> np.ndarray:
    """Truncated 3D solenoidal velocity spectrum with the same modulus on every
    retained mode but k = 0 (a flat, white spectrum up to the 2/3 cut-off), so
    every retained row of every axis carries energy.  Random phases and
    directions as in random_velocity_3d (same generator, same keys); built
    ``planes`` kz rows at a time so that 1024^3 grids stay within a few GB of
    temporaries; mean energy = ``energy``."""
    kc, c, h = truncation(n)
    u = np.empty((3, c, c, h), np.complex128)
    i = np.arange(c)
    kfull = np.where(i <= kc, i, i - c)
    e = 0.0
    for z0 in range(0, c, planes):
        kz, ky, kx = np.meshgrid(kfull[z0:z0 + planes], kfull, np.arange(h), indexing="ij")
        blk = _solenoidal_modes(kx, ky, kz, seed, lambda k, ksafe: np.ones_like(k))
        u[:, z0:z0 + planes] = blk
        e += float(np.sum(np.where(kx == 0, 1.0, 2.0) * 0.5 * (np.abs(blk) ** 2).sum(0)))
    if e > 0:
        u *= np.sqrt(energy / e)
    return u


def grid_coords(n: int):
    return 2.0 * np.pi * np.arange(n) / n


def taylor_green_3d(n: int) -> np.ndarray:
    """u = (sin x cos y cos z, -cos x sin y cos z, 0), layout (3, z, y, x)."""
    x = grid_coords(n)
    z3, y3, x3 = np.meshgrid(x, x, x, indexing="ij")
    u = np.zeros((3, n, n, n))
    u[0] = np.sin(x3) * np.cos(y3) * np.cos(z3)
    u[1] = -np.cos(x3) * np.sin(y3) * np.cos(z3)
    return u


def taylor_green_vorticity_2d(n: int) -> np.ndarray:
    """omega = 2 sin x sin y (the curl of u = (sin x cos y, -cos x sin y)),
    layout (y, x)."""
    x = grid_coords(n)
    y2, x2 = np.meshgrid(x, x, indexing="ij")
    return 2.0 * np.sin(x2) * np.sin(y2)


def abc_flow(n: int, A: float = 1.0, B: float = 1.0, C: float = 1.0) -> np.ndarray:
    """Arnold-Beltrami-Childress flow (curl u = u), layout (3, z, y, x)."""
    x = grid_coords(n)
    z3, y3, x3 = np.meshgrid(x, x, x, indexing="ij")
    return np.stack([A * np.sin(z3) + C * np.cos(y3),
                     B * np.sin(x3) + A * np.cos(z3),
                     C * np.sin(y3) + B * np.cos(x3)])


def shear_flow(n: int, k: int = 1) -> np.ndarray:
    """u = (sin(k y), 0, 0), layout (3, z, y, x)."""
    x = grid_coords(n)
    z3, y3, x3 = np.meshgrid(x, x, x, indexing="ij")
    u = np.zeros((3, n, n, n))
    u[0] = np.sin(k * y3)
    return u


def kolmogorov_forcing_2d(n: int, amp: float = 4.0, k: int = 4) -> np.ndarray:
    """Vorticity forcing amp * sin(k y), layout (y, x)."""
    x = grid_coords(n)
    y2, _ = np.meshgrid(x, x, indexing="ij")
    return amp * np.sin(k * y2)


def random_phys(shape, seed: int) -> np.ndarray:
    """White noise in [-1, 1) for tests of transforms (keyed by flat index)."""
    size = int(np.prod(shape))
    idx = np.arange(size, dtype=np.uint64)
    with np.errstate(over="ignore"):
        r = splitmix64(idx ^ splitmix64(np.uint64(seed + 12345)))
    u = (r >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return (2.0 * u - 1.0).reshape(shape)


def ensemble_sizes(count: int = 64, choices=(128, 256, 512), base: int = 1000):
    """Grid sizes of an ensemble: member i takes choices[splitmix64(base + i) mod len]."""
    r = splitmix64(np.arange(base, base + count, dtype=np.uint64))
    return [int(choices[int(v % np.uint64(len(choices)))]) for v in r]
