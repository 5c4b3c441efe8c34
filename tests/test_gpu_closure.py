"""GPU parity for the learned-closure pieces: the CNN kernels (forward,
gradients, Adam) against the FP64 oracle of oracle/closure_net.py, and the
device-side state/forcing hooks of the solver against the spectral oracle.

CNN tolerances.  Activations, pre-activations and weights are stored in
BF16 (unit roundoff u = 2^-9 ~ 1.95e-3), accumulation is FP32.  Each layer
adds a relative error of order u from its rounded inputs and weights; over
four layers that is a few u in the RMS sense: the forward output is held to
relative L2 1e-2 (~5 u), the weight and bias gradients to 3e-2 per layer
(the backward pass chains the rounded pre-activations through GELU' as well).
"""
import numpy as np
import pytest

from paper_1807_01769_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ns():
    from paper_1807_01769_gb300 import ns as mod

    return mod


@pytest.fixture(scope="module")
def cn():
    from oracle import closure_net

    return closure_net


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


def params(cn, seed):
    """He-scaled uniform weights and small biases from the seeded generator."""
    parts = []
    for li, (co, ci) in enumerate(cn.layer_shapes()):
        w = inputs.random_phys((co * ci * 9,), seed + 17 * li) * np.sqrt(6.0 / (9 * ci))
        b = 0.1 * inputs.random_phys((co,), seed + 17 * li + 5)
        parts += [w, b]
    return np.concatenate(parts).astype(np.float32)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("batch,h,w", [(1, 64, 64), (2, 64, 128), (3, 128, 64)])
def test_cnn_forward_matches_oracle(ns, cn, batch, h, w):
    p = params(cn, 100 + batch)
    x = inputs.random_phys((batch, h, w), 200 + batch)
    with ns.CNN(h, w, max_batch=3, seed=1) as net:
        net.set_params(p)
        np.testing.assert_array_equal(net.get_params(), p)
        xd, yd = dev(x), torch.empty((batch, h, w), dtype=torch.float32, device="cuda")
        net.forward(xd.data_ptr(), yd.data_ptr(), batch)
        torch.cuda.synchronize()
        y = yd.cpu().numpy()
    ref, _ = cn.forward(p.astype(np.float64), x)
    assert np.all(np.isfinite(y))
    assert rel(y, ref) < 1e-2, rel(y, ref)


def test_cnn_gradients_match_oracle(ns, cn):
    batch, h, w = 2, 64, 128
    p = params(cn, 300)
    x = inputs.random_phys((batch, h, w), 301)
    t = inputs.random_phys((batch, h, w), 302)
    with ns.CNN(h, w, max_batch=batch, seed=1) as net:
        net.set_params(p)
        xd, td = dev(x), dev(t)  # held: a temporary's memory would be reused by the next allocation
        g, loss = net.gradients(xd.data_ptr(), td.data_ptr(), batch)
    gref, lref = cn.gradients(p.astype(np.float64), x, t)
    assert abs(loss - lref) < 1e-2 * lref
    off = 0
    for co, ci in cn.layer_shapes():
        nw = co * ci * 9
        assert rel(g[off:off + nw], gref[off:off + nw]) < 3e-2, ("W", co, ci, rel(g[off:off + nw], gref[off:off + nw]))
        off += nw
        assert rel(g[off:off + co], gref[off:off + co]) < 3e-2, ("b", co, ci, rel(g[off:off + co], gref[off:off + co]))
        off += co


def test_cnn_adam_first_step(ns, cn):
    batch, h, w = 2, 64, 64
    p = params(cn, 400)
    x = inputs.random_phys((batch, h, w), 401)
    t = inputs.random_phys((batch, h, w), 402)
    lr = 1e-3
    with ns.CNN(h, w, max_batch=batch, seed=1) as net:
        net.set_params(p)
        xd, td = dev(x), dev(t)
        loss = net.train_step(xd.data_ptr(), td.data_ptr(), batch, lr)
        p1 = net.get_params()
    gref, lref = cn.gradients(p.astype(np.float64), x, t)
    pref, _, _ = cn.adam_step(p.astype(np.float64), gref, np.zeros_like(gref), np.zeros_like(gref), 1, lr)
    assert abs(loss - lref) < 1e-2 * lref
    d, dref = p1.astype(np.float64) - p, pref - p
    assert np.all(np.abs(d) <= lr * (1 + 1e-3))  # the first Adam step moves every parameter by at most lr
    big = np.abs(gref) > 0.05 * np.sqrt(np.mean(gref ** 2))
    agree = np.abs(d[big] - dref[big]) <= 1e-3 * lr + 1e-7
    assert agree.mean() > 0.995, agree.mean()


def test_cnn_tensor_core_path_equals_cuda_core_path(ns, cn):
    """The 32 -> 32 convolutions of widths that are multiples of 128 run on the
    tensor cores (tcgen05 implicit GEMM), the others on the CUDA cores.  The
    network is periodic and translation-equivariant, so a 256-wide input made
    of a 64-wide one tiled four times must give the tiled 64-wide output and
    gradients of the same network on the tiled batch: BF16 products are exact
    on both paths, only the FP32 summation order (and, where it flips a BF16
    rounding of an activation, that rounding) differs."""
    p = params(cn, 600)
    h = 64
    x = inputs.random_phys((2, h, 64), 601)
    t = inputs.random_phys((2, h, 64), 602)
    xt, tt = np.tile(x, (1, 1, 4)), np.tile(t, (1, 1, 4))
    with ns.CNN(h, 64, max_batch=2, seed=1) as a, ns.CNN(h, 256, max_batch=2, seed=1) as b:
        a.set_params(p)
        b.set_params(p)
        xd, xtd = dev(x), dev(xt)
        ya = torch.empty((2, h, 64), dtype=torch.float32, device="cuda")
        yb = torch.empty((2, h, 256), dtype=torch.float32, device="cuda")
        a.forward(xd.data_ptr(), ya.data_ptr(), 2)
        b.forward(xtd.data_ptr(), yb.data_ptr(), 2)
        torch.cuda.synchronize()
        ya, yb = ya.cpu().numpy(), yb.cpu().numpy()
        assert rel(yb, np.tile(ya, (1, 1, 4))) < 2e-3, rel(yb, np.tile(ya, (1, 1, 4)))
        td, ttd = dev(t), dev(tt)
        ga, la = a.gradients(xd.data_ptr(), td.data_ptr(), 2)
        gb, lb = b.gradients(xtd.data_ptr(), ttd.data_ptr(), 2)
    # the mean squared error over the tiled batch equals the untiled one
    assert abs(lb - la) < 1e-4 * la
    assert rel(gb, ga) < 3e-3, rel(gb, ga)


def test_cnn_training_fits_a_teacher(ns, cn):
    """Teacher-student: targets from the oracle network with fixed parameters;
    a differently initialised student trained by the GPU Adam loop fits them."""
    batch, h, w = 4, 64, 64
    teacher = params(cn, 500)
    x = inputs.random_phys((batch, h, w), 501)
    t, _ = cn.forward(teacher.astype(np.float64), x)
    t = t / np.std(t)
    xd, td = dev(x), dev(t)
    with ns.CNN(h, w, max_batch=batch, seed=7) as net:
        losses = [net.train_step(xd.data_ptr(), td.data_ptr(), batch, 2e-3) for _ in range(300)]
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])


def test_cnn_rejects_bad_shapes(ns):
    with pytest.raises(ns.NSError) as ei:
        ns.CNN(48, 64, 1)
    assert ei.value.code == ns.NS_EINVAL
    with ns.CNN(64, 64, 2) as net:
        x = torch.zeros((3, 64, 64), device="cuda")
        with pytest.raises(ns.NSError):
            net.forward(x.data_ptr(), x.data_ptr(), 3)


# ---------------------------------------------------------- solver hooks ---
@pytest.mark.parametrize("dim,n,prec,tol", [(2, 128, 0, 1e-12), (2, 256, 1, 2e-6), (3, 64, 1, 2e-6)])
def test_state_to_phys_device(ns, orc, dim, n, prec, tol):
    u = inputs.random_vorticity_2d(n, seed=3) if dim == 2 else inputs.random_velocity_3d(n, seed=3)
    with ns.Solver(dim, n, prec, nu=1e-3, dt=1e-3) as s:
        s.set_state_spectral(u)
        buf = torch.empty(orc.phys_shape(dim, n), dtype=torch.float64, device="cuda")
        ns._check(ns.lib.ns_state_to_phys_device(s.state, ns.ctypes.c_void_p(buf.data_ptr())), s.state)
        s.sync()
        got = buf.cpu().numpy()
    ref = orc.state_to_phys(dim, n, u)
    assert rel(got, ref) < tol


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 1e-5)])
def test_forcing_set_on_device_matches_oracle(ns, orc, prec, tol):
    n, nu, dt, steps = 128, 1e-3, 1e-3, 10
    u = inputs.random_vorticity_2d(n, seed=4)
    f_phys = inputs.kolmogorov_forcing_2d(n)
    f_spec = orc.phys_to_state(2, n, f_phys)
    ref = orc.step(2, n, nu, dt, steps, u, forcing=f_spec)
    with ns.Solver(2, n, prec, nu=nu, dt=dt) as s:
        s.set_state_spectral(u)
        s.step(2)  # a step graph without forcing exists before the forcing arrives
        s.set_state_spectral(u)
        fd = torch.from_numpy(f_phys).cuda()
        ns._check(ns.lib.ns_set_forcing_phys_device(s.state, ns.ctypes.c_void_p(fd.data_ptr())), s.state)
        s.step(steps)
        got = s.get_state_spectral()
    w = np.where(np.arange(u.shape[-1]) == 0, 1.0, 2.0)
    err = np.sqrt(np.sum(w * np.abs(got - ref) ** 2) / np.sum(w * np.abs(ref) ** 2))
    assert err < tol, err


def test_conversion_helpers(ns):
    n = 5000
    src = torch.linspace(-3, 3, n, dtype=torch.float64, device="cuda")
    f = torch.empty(n, dtype=torch.float32, device="cuda")
    ns.f64_to_f32(src.data_ptr(), f.data_ptr(), n, 0.5)
    base = torch.full((n,), 2.0, dtype=torch.float64, device="cuda")
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    ns.f32_axpy_f64(f.data_ptr(), base.data_ptr(), out.data_ptr(), n, 4.0)
    torch.cuda.synchronize()
    s = np.linspace(-3, 3, n)
    np.testing.assert_array_equal(f.cpu().numpy(), (0.5 * s).astype(np.float32))
    f32 = (0.5 * s).astype(np.float32).astype(np.float64)
    np.testing.assert_allclose(out.cpu().numpy(), 2.0 + 4.0 * f32, rtol=0, atol=1e-15)


# ------------------------------------------------- closure, end to end ---
def test_closure_gains_over_the_plain_coarse_solve(ns):
    """Forced Kolmogorov flow (4 sin 4y, nu = 1e-3), fine 512^2 runs filtered
    to 128^2 (seeds 0..3, 40 snapshots each), 400 Adam steps; on the held-out
    seed 100 the trained network must (a) predict the closure target better
    than the plain coarse solve's implicit zero (skill > 0.2) and (b) keep the
    closed 128^2 run nearer to the filtered 512^2 run than the plain 128^2
    run: smaller vorticity error at t = 0.5 and a smaller shell-spectrum error
    at t = 0.5 and t = 2."""
    from paper_1807_01769_gb300 import closure as C

    cfg = C.KolmogorovConfig(n_fine=512, n_coarse=128, dt_coarse=4e-3, t_spin=2.0, snap_every=0.05,
                             snaps_per_seed=40, train_seeds=(0, 1, 2, 3))
    X, T, _ = C.generate(cfg, cfg.train_seeds)
    assert np.all(np.isfinite(X)) and np.all(np.isfinite(T))
    tr = C.train(X, T, steps=400, batch=8, lr=2e-3)
    try:
        assert tr.losses[-1][1] < 0.5 * tr.losses[0][1]
        Xe, Te, _ = C.generate(C.KolmogorovConfig(**{**C.asdict(cfg), "snaps_per_seed": 10}), (100,))
        prior = C.a_priori(tr, Xe, Te)
        assert prior["skill"] > 0.2, prior
        rows = C.a_posteriori(cfg, tr, 100, 2.0, 0.5)["rows"]
        assert not any(r["fell_back"] for r in rows)
        assert rows[0]["err_closure"] < rows[0]["err_plain"], rows[0]
        assert rows[0]["spec_err_closure"] < rows[0]["spec_err_plain"], rows[0]
        assert rows[-1]["spec_err_closure"] < rows[-1]["spec_err_plain"], rows[-1]
    finally:
        tr.net.close()


@pytest.mark.parametrize("mode", ["fine", "coarse"])
def test_closure_fallback_hands_over_to_the_plain_solve(ns, mode):
    """A closed run that blows up (here: a network whose output is scaled by
    1e8) restores its last good state and continues without the network: by
    default as the plain fine-grid solve restarted from that state prolonged
    to the fine grid, its coarse view the fine state filtered back; with
    fallback="coarse" as the plain coarse solve.  Either way it must equal,
    bit for bit, the plain solve started from the same state."""
    from paper_1807_01769_gb300 import closure as C

    cfg = C.KolmogorovConfig(n_fine=256, n_coarse=128, dt_coarse=4e-3)
    w0 = inputs.random_vorticity_2d(128, seed=9, k0=8.0, energy=0.5)
    net = ns.CNN(128, 128, 1, seed=3)
    tr = C.Trained(net, x_scale=6.0, t_scale=1e8)
    try:
        cs = C.ClosureSolver(cfg, tr, check_every=5, fallback=mode)
        try:
            cs.set_state_spectral(w0)
            cs.step(20)  # the check after 5 steps fails: the last good state is w0
            assert cs.fell_back and cs.on_fine == (mode == "fine")
            got = cs.get_state_spectral()
            e, om = cs.diagnostics()
            assert np.all(np.isfinite(got)) and np.isfinite(e) and np.isfinite(om)
        finally:
            cs.close()
        if mode == "fine":
            with C.fine_solver(cfg) as f:
                f.set_state_spectral(C.prolong_2d(w0, 128, 256))
                f.step(15 * cfg.ratio)
                ref = C.restrict_2d(f.get_state_spectral(), 256, 128)
        else:
            with C.coarse_solver(cfg) as c:
                c.set_state_spectral(w0)
                c.step(15)
                ref = c.get_state_spectral()
        assert np.array_equal(got, ref)
    finally:
        net.close()


def test_closure_graph_replay_equals_eager_steps(ns):
    """One corrected step captured into a CUDA graph and replayed gives the
    same state, bit for bit, as the same steps launched one by one."""
    from paper_1807_01769_gb300 import closure as C

    cfg = C.KolmogorovConfig(n_fine=256, n_coarse=128, dt_coarse=4e-3)
    w0 = inputs.random_vorticity_2d(128, seed=9, k0=8.0, energy=0.5)
    net = ns.CNN(128, 128, 1, seed=3)
    tr = C.Trained(net, x_scale=6.0, t_scale=2.0)
    out = []
    try:
        for use_graph in (True, False):
            cs = C.ClosureSolver(cfg, tr, check_every=7, use_graph=use_graph)
            try:
                cs.set_state_spectral(w0)
                cs.step(20)
                out.append(cs.get_state_spectral())
                assert not cs.fell_back
            finally:
                cs.close()
    finally:
        net.close()
    np.testing.assert_array_equal(out[0], out[1])
    assert np.any(out[0] != w0)