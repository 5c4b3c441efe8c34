"""GPU parity of the tensor-core precision NS_FP32_TC (3D): the x-line
transforms run as split-BF16 GEMMs on the tensor cores, everything else as in
NS_FP32.  Compared with the FP64 oracle on the canonical spectral layout.

Tolerances: one transform carries about 2^-16 relative error per product (hi*lo
and lo*hi keep 16 significant bits of each operand; the dropped lo*lo term and
the rounding of lo are each below 2^-16 of the product), summed over a few dozen
terms per output with random signs; six inverse and three forward transforms
per right-hand side leave a relative L2 error of order 1e-5.  The right-hand
side is checked at 1e-4, ten 64^3 RK4 steps against the 1e-3 target for this
precision, and the energy of the 512^3 run against the FP32 path at 1e-5.
"""
import numpy as np
import pytest

from paper_1807_01769_gb300 import inputs

pytestmark = pytest.mark.gpu

FP32, TC = 1, 2
TOL_RHS_TC = 1e-4
TOL_STEPS_TC = 1e-3


@pytest.fixture(scope="module")
def ns():
    from paper_1807_01769_gb300 import ns as mod

    return mod


def rel_l2(a, b):
    w = np.full(b.shape[-1], 2.0)
    w[0] = 1.0
    return float(np.sqrt(np.sum(w * np.abs(a - b) ** 2) / np.sum(w * np.abs(b) ** 2)))


def ic(n, seed=0):
    return inputs.random_velocity_3d(n, seed=seed, k0=4.0, a=2.0, energy=0.5)


def low_modes(u, n_from, n_to):
    kc_f, c_f, h_f = inputs.truncation(n_from)
    kc_t, c_t, h_t = inputs.truncation(n_to)
    i = np.arange(c_t)
    k = np.where(i <= kc_t, i, i - c_t)
    j = np.where(k >= 0, k, k + c_f)
    return u[:, j][:, :, j][..., :h_t]


def embed(u_small, n_small, n_big):
    kc_s, c_s, h_s = inputs.truncation(n_small)
    kc_b, c_b, h_b = inputs.truncation(n_big)
    out = np.zeros((3, c_b, c_b, h_b), np.complex128)
    i = np.arange(c_s)
    k = np.where(i <= kc_s, i, i - c_s)
    j = np.where(k >= 0, k, k + c_b)
    for a in range(3):
        for p, jz in enumerate(j):
            out[a, jz, j, :h_s] = u_small[a, p]
    return out


@pytest.mark.parametrize("n", [64, 128, 256])
def test_tc_rhs_matches_oracle(ns, orc, n):
    u = ic(n, seed=3)
    with ns.Solver(3, n, TC, nu=1e-3, dt=1e-3) as s:
        s.set_state_spectral(u)
        got = s.eval_rhs()
        ref = orc.rhs(3, n, s.get_state_spectral())
    err = rel_l2(got, ref)
    assert err < TOL_RHS_TC, err
    assert err > 1e-9  # the tensor-core path really ran (FP32 ALU error is ~1e-7)


def test_tc_rhs_with_forcing(ns, orc):
    n = 64
    u = ic(n, seed=4)
    f = orc.state_to_phys(3, n, 3.0 * ic(n, seed=5))
    with ns.Solver(3, n, TC, nu=1e-3, dt=1e-3, forcing_phys=f) as s:
        s.set_state_spectral(u)
        got = s.eval_rhs()
        ref = orc.rhs(3, n, s.get_state_spectral(), forcing=orc.phys_to_state(3, n, f))
    assert rel_l2(got, ref) < TOL_RHS_TC


def test_tc_ten_steps_64_within_target(ns, orc):
    # random-phase solenoidal field, nu = 2e-3, dt = 1e-3, 10 Lawson RK4 steps
    n, nu, dt, steps = 64, 2e-3, 1e-3, 10
    u0 = ic(n, seed=1)
    with ns.Solver(3, n, TC, nu=nu, dt=dt) as s:
        s.set_state_spectral(u0)
        s.step(steps)
        got = s.get_state_spectral()
    ref = orc.step(3, n, nu, dt, steps, u0)
    err = rel_l2(got, ref)
    assert err < TOL_STEPS_TC, err


def test_tc_rhs_512_band_limited_equals_oracle_64(ns, orc):
    # the bench grid: a field with only 64^3 modes, whose dealiased product is
    # exact on both grids
    m, n = 64, 512
    u_small = ic(m, seed=13)
    ref = orc.rhs(3, m, u_small)
    with ns.Solver(3, n, TC, nu=2e-3, dt=1e-3) as s:
        s.set_state_spectral(embed(u_small, m, n))
        got = s.eval_rhs()
    assert rel_l2(low_modes(got, n, m), ref) < TOL_RHS_TC


def test_tc_bench_workload_512_20_steps(ns, orc):
    n, nu, dt, steps = 512, 2e-3, 1e-3, 20
    with ns.Solver(3, n, TC, nu=nu, dt=dt) as s:
        s.set_state_spectral(ic(n, seed=0))
        s.step(steps)
        s.sync()
        e, om = s.diagnostics()
        u = s.get_state_spectral()
    m = 64
    ref = orc.step(3, m, nu, dt, steps, ic(m, seed=0))
    assert rel_l2(low_modes(u, n, m), ref) < TOL_STEPS_TC
    re, rom = orc.diagnostics(3, m, ref)
    assert abs(e - re) < 1e-5 * re and abs(om - rom) < 1e-5 * rom


def test_tc_is_deterministic_and_chunk_invariant(ns, monkeypatch):
    n = 128
    u0 = ic(n, seed=12)
    out = []
    for chunks in ("1", "1", "8"):
        monkeypatch.setenv("NS_ZCHUNKS", chunks)
        with ns.Solver(3, n, TC, nu=2e-3, dt=1e-3) as s:
            s.set_state_spectral(u0)
            s.step(3)
            out.append(s.get_state_spectral())
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_tc_cfl_maxima_match_fp32(ns):
    # the x pass maxima of |u_i| set the CFL step: same dt as the FP32 path to
    # the accuracy of the velocity values
    n = 64
    u0 = ic(n, seed=2)
    t = []
    for prec in (FP32, TC):
        with ns.Solver(3, n, prec, nu=2e-3, dt=1e-2) as s:
            s.set_state_spectral(u0)
            s.set_cfl(0.5)
            s.step(1)
            s.sync()
            t.append(s.time()[0])
    assert abs(t[1] - t[0]) < 1e-5 * t[0]
