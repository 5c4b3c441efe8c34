"""CPU model of the arithmetic the tensor-core x pass (precision NS_FP32_TC)
is built on, checked against numpy's FFT: the two-GEMM (four-step) form of a
length-N DFT with its index maps, the real-block DFT matrices, the pairing of
two real fields into one complex line (inverse: Hermitian extension; forward:
the conjugation trick and the split with the partner mode), and the error
level of BF16 hi + lo operands with three products and FP32 accumulation
that the GPU tolerances are derived from.  No GPU and no library code: the
formulas are restated here from their definitions."""
import numpy as np
import pytest

PLANS = {64: (8, 8), 128: (8, 16), 256: (16, 16), 512: (16, 32)}


def real_block(R):
    """K-by-N real matrix of the length-R DFT with exponent +2 pi i a c / R:
    rows (p, a) = real / imaginary input part, columns (q, c) likewise."""
    a = np.arange(R)
    th = 2 * np.pi * np.outer(a, a) / R
    C, S = np.cos(th), np.sin(th)
    return np.block([[C, S], [-S, C]])


def two_gemm_dft(x, R1, R2, gemm=lambda A, B: A @ B):
    """X[c + R1 d] = sum_n x[n] exp(+2 pi i n k / N) for lines x[..., N] via
    stage A (DFT-R1 over a, n = R2 a + b), twiddle w^(b c), stage B (DFT-R2 over b)."""
    N = R1 * R2
    lines = x.reshape(-1, N)
    m = lines.shape[0]
    # stage A rows (line, b): inputs x[R2 a + b], a = 0..R1-1, as [re | im]
    xa = lines.reshape(m, R1, R2).transpose(0, 2, 1)  # [line][b][a]
    A = np.concatenate([xa.real, xa.imag], axis=-1).reshape(m * R2, 2 * R1)
    Y = gemm(A, real_block(R1)).reshape(m, R2, 2 * R1)
    Y = Y[..., :R1] + 1j * Y[..., R1:]  # [line][b][c]
    b = np.arange(R2)[:, None]
    c = np.arange(R1)[None, :]
    Y = Y * np.exp(2j * np.pi * b * c / N)
    # stage B rows (line, c): inputs Y'[b][c], b = 0..R2-1
    Yb = Y.transpose(0, 2, 1)  # [line][c][b]
    B = np.concatenate([Yb.real, Yb.imag], axis=-1).reshape(m * R1, 2 * R2)
    X = gemm(B, real_block(R2)).reshape(m, R1, 2 * R2)
    X = X[..., :R2] + 1j * X[..., R2:]  # [line][c][d], k = c + R1 d
    return X.transpose(0, 2, 1).reshape(x.shape)


@pytest.mark.parametrize("N", sorted(PLANS))
def test_two_gemm_form_is_the_dft(N):
    R1, R2 = PLANS[N]
    rng = np.random.default_rng(N)
    x = rng.standard_normal((5, N)) + 1j * rng.standard_normal((5, N))
    ref = np.fft.ifft(x, axis=-1) * N  # exponent +
    assert np.allclose(two_gemm_dft(x, R1, R2), ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def hermitian_pair(Xa, Xb, N):
    """z's spectrum Z from two half spectra (modes 0..kc): Z[k] = Xa + i Xb,
    Z[N-k] = conj(Xa) + i conj(Xb), modes above kc zero, Im of mode 0 dropped."""
    kc = Xa.shape[-1] - 1
    Xa, Xb = Xa.copy(), Xb.copy()
    Xa[..., 0] = Xa[..., 0].real
    Xb[..., 0] = Xb[..., 0].real
    Z = np.zeros(Xa.shape[:-1] + (N,), complex)
    Z[..., : kc + 1] = Xa + 1j * Xb
    Z[..., N - kc:] = (np.conj(Xa) + 1j * np.conj(Xb))[..., kc:0:-1]
    return Z


@pytest.mark.parametrize("N", sorted(PLANS))
def test_paired_inverse_gives_both_real_lines(N):
    R1, R2 = PLANS[N]
    kc = (N - 1) // 3
    rng = np.random.default_rng(7 + N)
    Xa = rng.standard_normal((3, kc + 1)) + 1j * rng.standard_normal((3, kc + 1))
    Xb = rng.standard_normal((3, kc + 1)) + 1j * rng.standard_normal((3, kc + 1))
    z = two_gemm_dft(hermitian_pair(Xa, Xb, N), R1, R2)
    # each real line: the unnormalised c2r of its half spectrum (Im of mode 0 dropped)
    for X, part in ((Xa, z.real), (Xb, z.imag)):
        full = np.zeros((3, N // 2 + 1), complex)
        full[:, : kc + 1] = X
        full[:, 0] = full[:, 0].real
        ref = np.fft.irfft(full, n=N, axis=-1) * N
        assert np.allclose(part, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


@pytest.mark.parametrize("N", sorted(PLANS))
def test_paired_forward_conjugation_and_split(N):
    """G = DFT_+(conj(y_a + i y_b)); with Z = conj G: Y_a = (Z[k] + conj Z[N-k]) / 2,
    Y_b = (Z[k] - conj Z[N-k]) / (2 i) equal the r2c of y_a and y_b."""
    R1, R2 = PLANS[N]
    kc = (N - 1) // 3
    rng = np.random.default_rng(11 + N)
    ya, yb = rng.standard_normal((2, 4, N))
    G = two_gemm_dft(np.conj(ya + 1j * yb), R1, R2)
    k = np.arange(kc + 1)
    g, h = G[:, k], G[:, (N - k) % N]  # h = G[N - k] (the partner mode)
    Ya = 0.5 * ((g.real + h.real) + 1j * (h.imag - g.imag))
    Yb = 0.5 * (-(g.imag + h.imag) + 1j * (h.real - g.real))
    for Y, y in ((Ya, ya), (Yb, yb)):
        ref = np.fft.rfft(y, axis=-1)[:, : kc + 1]
        assert np.allclose(Y, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def bf16_rn(x):
    """Round float32 values to the nearest BF16 (ties to even), returned as float32."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32)


def split(x):
    hi = bf16_rn(x)
    lo = bf16_rn(np.float32(x) - hi)
    return hi, lo


def split3_gemm(A, B):
    """hi*hi + hi*lo + lo*hi with BF16 parts, products exact, sums in FP32."""
    ah, al = split(A.astype(np.float32))
    bh, bl = split(B.astype(np.float32))
    f = lambda P, Q: (P.astype(np.float64) @ Q.astype(np.float64)).astype(np.float32)
    return (f(ah, bh) + f(ah, bl) + f(al, bh)).astype(np.float64)


def test_bf16_split_reconstructs_to_sixteen_bits():
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(100000) * np.exp(rng.uniform(-20, 20, 100000))).astype(np.float32)
    hi, lo = split(x)
    assert np.all(np.abs(lo) <= 2.0 ** -8 * np.abs(x) * (1 + 1e-6))
    rel = np.abs((hi.astype(np.float64) + lo) - x) / np.abs(x)
    assert rel.max() <= 2.0 ** -16


@pytest.mark.parametrize("N", [256, 512])
def test_split_precision_dft_error_level(N):
    """The two-GEMM DFT with split-BF16 operands stays within the ~1e-5 the
    GPU tolerances assume, and is clearly coarser than FP64 (the model really
    rounds)."""
    R1, R2 = PLANS[N]
    rng = np.random.default_rng(5 + N)
    x = rng.standard_normal((64, N)) + 1j * rng.standard_normal((64, N))
    ref = np.fft.ifft(x, axis=-1) * N
    got = two_gemm_dft(x, R1, R2, gemm=split3_gemm)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert 1e-8 < err < 1e-5, err
    # one product without the lo terms (plain BF16) is far worse: the lo terms carry the accuracy
    plain = two_gemm_dft(x, R1, R2, gemm=lambda A, B: (bf16_rn(A.astype(np.float32)).astype(np.float64)
                                                       @ bf16_rn(B.astype(np.float32)).astype(np.float64)))
    assert np.linalg.norm(plain - ref) / np.linalg.norm(ref) > 100 * err
