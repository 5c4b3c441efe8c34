"""Pins of the oracle's transforms against definitions that do not use it:
brute-force DFT sums, numpy's independent FFT, Parseval, single modes."""
import numpy as np
import pytest

from paper_1807_01769_gb300 import inputs


def brute_dft(x, sign):
    n = x.size
    j = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(j, j) / n) @ x


@pytest.mark.parametrize("n", [2, 4, 8, 16])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft1d_vs_brute_force(orc, n, sign):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = brute_dft(x, sign)
    got = orc.fft1d(x, sign)
    assert np.abs(got - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("n", [64, 1024])
def test_fft1d_vs_numpy(orc, n):
    rng = np.random.default_rng(7)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.abs(orc.fft1d(x, -1) - np.fft.fft(x)).max() < 1e-11
    assert np.abs(orc.fft1d(x, 1) - n * np.fft.ifft(x)).max() < 1e-11


def brute_rfftn(u):
    """u_hat(k) = N^-d sum_x u(x) exp(-i k.x), kx = 0..N/2 (definition)."""
    n = u.shape[0]
    d = u.ndim
    j = np.arange(n)
    f = np.exp(-2j * np.pi * np.outer(j, j) / n)  # [k, x]
    out = u.astype(np.complex128)
    # apply the 1D DFT matrix along every axis (a plain sum per axis)
    for ax in range(d):
        out = np.moveaxis(np.tensordot(f, np.moveaxis(out, ax, 0), axes=(1, 0)), 0, ax)
    return out[..., : n // 2 + 1] / n ** d


@pytest.mark.parametrize("shape", [(8, 8), (16, 16), (8, 8, 8)])
def test_rfftn_vs_brute_force(orc, shape):
    u = inputs.random_phys(shape, seed=3)
    got = orc.rfftn(len(shape), shape[0], u)
    ref = brute_rfftn(u)
    assert np.abs(got - ref).max() < 1e-14


@pytest.mark.parametrize("dim,n", [(2, 64), (3, 32)])
def test_rfftn_vs_numpy_and_roundtrip(orc, dim, n):
    u = inputs.random_phys((n,) * dim, seed=11)
    s = orc.rfftn(dim, n, u)
    assert np.abs(s - np.fft.rfftn(u) / n ** dim).max() < 1e-14
    back = orc.irfftn(dim, n, s * n ** dim / n ** dim)
    # irfftn is unnormalised and rfftn normalised: the pair is the identity
    assert np.abs(back - u).max() < 1e-12
    # Parseval: mean of u^2 = sum over the full spectrum of |u_hat|^2
    w = np.ones(n // 2 + 1) * 2.0
    w[0] = 1.0
    w[-1] = 1.0
    assert np.isclose((u ** 2).mean(), (w * np.abs(s) ** 2).sum(), rtol=1e-12)


def test_single_mode_gives_delta(orc):
    n = 16
    x = inputs.grid_coords(n)
    y2, x2 = np.meshgrid(x, x, indexing="ij")
    u = np.cos(3 * x2 - 2 * y2)
    s = orc.rfftn(2, n, u)
    ref = np.zeros_like(s)
    ref[(-2) % n, 3] = 0.5  # cos = (e^{i k.x} + e^{-i k.x})/2, kx >= 0 half keeps one
    assert np.abs(s - ref).max() < 1e-15


def test_irfftn_uses_real_part_of_self_conjugate_modes(orc):
    # Imaginary parts on kx = 0 / kx = N/2 that break Hermitian symmetry are
    # discarded by "take the real part" (the stated c2r convention).
    n = 8
    s = np.zeros((n, n // 2 + 1), np.complex128)
    s[0, 0] = 1.0 + 5.0j
    u = orc.irfftn(2, n, s)
    assert np.allclose(u, 1.0, atol=1e-15)
