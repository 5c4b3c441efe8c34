"""Batched ensembles of 2D runs of uneven sizes: every member must equal (bit
for bit) the same run advanced alone by ns_step, for any schedule, and match
the FP64 oracle within the path's tolerance."""
import numpy as np
import pytest

from paper_1807_01769_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1


@pytest.fixture(scope="module")
def ns():
    from paper_1807_01769_gb300 import ns as mod

    return mod


def rel_l2(a, b):
    w = np.full(b.shape[-1], 2.0)
    w[0] = 1.0
    return float(np.sqrt(np.sum(w * np.abs(a - b) ** 2) / np.sum(w * np.abs(b) ** 2)))


def ic(n, seed):
    return inputs.random_vorticity_2d(n, seed=seed, k0=8.0, a=2.0, energy=0.5)


def single(ns, n, prec, nu, dt, steps, u0):
    with ns.Solver(2, n, prec, nu=nu, dt=dt) as s:
        s.set_state_spectral(u0)
        s.step(steps)
        return s.get_state_spectral()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_members_bitwise_equal_single_runs_for_every_schedule(ns, prec):
    sizes = [128, 256, 64, 512, 128, 256]
    nu, dt, steps = 5e-4, 5e-4, 5
    u0 = [ic(n, seed) for seed, n in enumerate(sizes)]
    ref = [single(ns, n, prec, nu, dt, steps, u) for n, u in zip(sizes, u0)]
    with ns.Ensemble(sizes, prec, nu=nu, dt=dt, autotune=True) as e:
        yt, xw = e.tiles()
        assert yt in (256, 512) and xw in (4, 8)
        # the autotuned schedule, then every tile shape with several grid and
        # order settings
        cases = [(None, None)] + [((yt, xw), sched) for yt in (256, 512) for xw in (4, 8)
                                  for sched in [(2, 1, 0), (8, 4, 1), (1, 2, 1)]]
        for tiles, sched in cases:
            if tiles is not None:
                e.set_tiles(*tiles)
                e.set_schedule(*sched)
            for m, u in enumerate(u0):
                e.set_state_spectral(m, u)
            e.step(steps)
            for m in range(len(sizes)):
                assert np.array_equal(e.get_state_spectral(m), ref[m]), (tiles, sched, m)
        with pytest.raises(ns.NSError):
            e.set_tiles(384, 4)


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_fused_form_equals_single_runs(ns, prec):
    """One cooperative launch per RK stage (x pass, grid-wide barrier, fused y
    pass) gives every member bit for bit the result of its own ns_step run,
    for every allowed block count and both task orders."""
    sizes = [128, 256, 64, 512, 128, 256]
    nu, dt, steps = 5e-4, 5e-4, 5
    u0 = [ic(n, seed) for seed, n in enumerate(sizes)]
    ref = [single(ns, n, prec, nu, dt, steps, u) for n, u in zip(sizes, u0)]
    with ns.Ensemble(sizes, prec, nu=nu, dt=dt, autotune=False) as e:
        f, fmax = e.fused()
        assert f == 0 and fmax >= 1
        for bpsm in sorted({1, fmax}):
            for order in (0, 1):
                e.set_fused(bpsm)
                e.set_schedule(2, 2, order)
                assert e.fused() == (bpsm, fmax) and e.tiles() == (256, 8)
                for m, u in enumerate(u0):
                    e.set_state_spectral(m, u)
                e.step(steps)
                e.sync()  # the barrier's bounded waits all ended in time
                for m in range(len(sizes)):
                    assert np.array_equal(e.get_state_spectral(m), ref[m]), (bpsm, order, m)
        with pytest.raises(ns.NSError):
            e.set_fused(fmax + 1)
        with pytest.raises(ns.NSError):
            e.set_fused(-1)
        e.set_tiles(256, 4)
        assert e.fused()[0] == 0


def test_members_match_oracle(ns, orc):
    sizes = [64, 128]
    nu, dt, steps = 1e-3, 1e-3, 20
    u0 = [ic(n, 3 + i) for i, n in enumerate(sizes)]
    with ns.Ensemble(sizes, FP64, nu=nu, dt=dt, autotune=False) as e:
        for m, u in enumerate(u0):
            e.set_state_spectral(m, u)
        e.step(steps)
        for m, n in enumerate(sizes):
            assert rel_l2(e.get_state_spectral(m), orc.step(2, n, nu, dt, steps, u0[m])) < 1e-11
        en, om = e.diagnostics()
    for m, n in enumerate(sizes):
        re, rom = orc.diagnostics(2, n, orc.step(2, n, nu, dt, steps, u0[m]))
        assert abs(en[m] - re) < 1e-12 * re and abs(om[m] - rom) < 1e-12 * rom


def test_full_ensemble_configuration(ns, orc):
    # 64 runs, sizes uniform in {128, 256, 512}, seeds 0..63, spectrum peaked at
    # k = 8, nu = dt = 5e-4, 200 steps; checked member by member where cheap
    sizes = inputs.ensemble_sizes(64)
    assert set(sizes) == {128, 256, 512}
    nu, dt, steps = 5e-4, 5e-4, 200
    u0 = [ic(n, seed) for seed, n in enumerate(sizes)]
    with ns.Ensemble(sizes, FP32, nu=nu, dt=dt, autotune=True) as e:
        for m, u in enumerate(u0):
            e.set_state_spectral(m, u)
        e.step(steps)
        en, om = e.diagnostics()
        checks = {}
        for n in (128, 256, 512):
            m = sizes.index(n)
            checks[m] = e.get_state_spectral(m)
    assert np.all(np.isfinite(en)) and np.all(en < 0.5) and np.all(en > 0.4)
    for m, got in checks.items():
        assert np.array_equal(got, single(ns, sizes[m], FP32, nu, dt, steps, u0[m]))
    m = sizes.index(128)
    assert rel_l2(checks[m], orc.step(2, 128, nu, dt, steps, u0[m])) < 1e-5


def test_all_64_members_bitwise_under_mixed_schedules(ns):
    # many members of different N per block and per warp: catches any sharing
    # of shared memory between units of different grids
    sizes = inputs.ensemble_sizes(64)
    nu, dt, steps = 5e-4, 5e-4, 20
    u0 = [ic(n, seed) for seed, n in enumerate(sizes)]
    ref = [single(ns, n, FP32, nu, dt, steps, u) for n, u in zip(sizes, u0)]
    with ns.Ensemble(sizes, FP32, nu=nu, dt=dt, autotune=False) as e:
        for tiles, sched in [((256, 4), (4, 2, 0)), ((512, 8), (8, 4, 1)), ((512, 4), (1, 1, 0)), ("fused", (1, 1, 1))]:
            if tiles == "fused":
                e.set_fused(1)
            else:
                e.set_tiles(*tiles)
            e.set_schedule(*sched)
            for m, u in enumerate(u0):
                e.set_state_spectral(m, u)
            e.step(steps)
            e.sync()
            bad = [m for m in range(len(sizes)) if not np.array_equal(e.get_state_spectral(m), ref[m])]
            assert not bad, (tiles, sched, bad[:8])
