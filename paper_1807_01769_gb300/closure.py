"""Learned closure for the coarse 2D vorticity solve (an extension: the paper
has no learned model; its 2D solver and Kolmogorov-type forcing are in the
2D benchmark and forcing sections).

The coarse solve advances the truncated vorticity of an N_c^2 grid; the
fine solve (N_f^2, same nu, same forcing) is the reference.  With the spectral
cut-off filter P (keep the modes the coarse grid retains) and the nonlinear
tendency N(omega) = -u . grad omega + F of the library (``ns_eval_rhs``),
the closure target is

    tau = P N_f(omega_f) - N_c(P omega_f),

the part of the filtered fine tendency the coarse grid cannot form itself.
The network maps the coarse vorticity (physical, normalised) to tau
(physical, normalised); during a closed run the prediction enters the coarse
solve as an additional forcing, refreshed before every step (held fixed
within one RK4 step).

Everything on the GPU runs through the library's kernels: the solver steps,
``ns_eval_rhs``, the device-side state/forcing hooks and the CNN forward,
backward and Adam kernels.  The host only selects modes (restriction of a
truncated spectrum), subtracts two tendencies while preparing training data
and shuffles snapshot order.

Fallback: a closed run checks the coarse enstrophy every ``check_every``
steps; if it is not finite or exceeds ``blowup`` times its starting value,
the run restores the last good state and continues without the network:
by default as the plain fine-grid solve, restarted from the last good coarse
state prolonged to the fine grid (zero padding of the modes the coarse grid
lacks), with the coarse view of the run the fine state filtered back to the
coarse modes; with ``fallback="coarse"`` as the plain coarse solve.
``fell_back`` is set either way.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time
from dataclasses import asdict, dataclass, field

import numpy as np

from . import inputs
from . import ns

FP32 = ns.NS_FP32


@dataclass
class KolmogorovConfig:
    n_fine: int = 2048
    n_coarse: int = 256
    nu: float = 1e-3
    dt_coarse: float = 2e-3
    amp: float = 4.0          # vorticity forcing amp * sin(kf y)
    kf: int = 4
    ic_k0: float = 8.0        # initial field: random phases, E(k) ~ k^4 exp(-(k/k0)^2), mean energy ic_energy
    ic_energy: float = 0.5
    t_spin: float = 4.0       # spin-up before the first snapshot
    snap_every: float = 0.05
    snaps_per_seed: int = 125
    train_seeds: tuple = tuple(range(16))
    eval_seed: int = 100

    @property
    def ratio(self) -> int:
        return self.n_fine // self.n_coarse

    @property
    def dt_fine(self) -> float:
        return self.dt_coarse / self.ratio

    def steps(self, t: float, fine: bool) -> int:
        dt = self.dt_fine if fine else self.dt_coarse
        return int(round(t / dt))


def restrict_2d(spec: np.ndarray, n_from: int, n_to: int) -> np.ndarray:
    """Spectral cut-off filter: the modes of an n_to grid taken out of a
    truncated (c, h) spectrum of an n_from grid (index selection only)."""
    kc_t, c_t, h_t = inputs.truncation(n_to)
    _, c_f, _ = inputs.truncation(n_from)
    i = np.arange(c_t)
    k = np.where(i <= kc_t, i, i - c_t)
    j = np.where(k >= 0, k, k + c_f)
    return np.ascontiguousarray(spec[j][:, :h_t])


def prolong_2d(spec: np.ndarray, n_from: int, n_to: int) -> np.ndarray:
    """The truncated (c, h) spectrum of an n_from grid placed into the
    truncated spectrum of a finer n_to grid, zero on every mode the coarse
    grid does not hold (index selection only; restrict_2d undoes it)."""
    kc_f, c_f, h_f = inputs.truncation(n_from)
    kc_t, c_t, h_t = inputs.truncation(n_to)
    out = np.zeros((c_t, h_t), np.complex128)
    i = np.arange(c_f)
    k = np.where(i <= kc_f, i, i - c_f)
    j = np.where(k >= 0, k, k + c_t)
    out[j, :h_f] = spec
    return out


def forcing(cfg: KolmogorovConfig, n: int) -> np.ndarray:
    return inputs.kolmogorov_forcing_2d(n, amp=cfg.amp, k=cfg.kf)


def fine_solver(cfg: KolmogorovConfig) -> ns.Solver:
    return ns.Solver(2, cfg.n_fine, FP32, nu=cfg.nu, dt=cfg.dt_fine, forcing_phys=forcing(cfg, cfg.n_fine))


def coarse_solver(cfg: KolmogorovConfig) -> ns.Solver:
    return ns.Solver(2, cfg.n_coarse, FP32, nu=cfg.nu, dt=cfg.dt_coarse, forcing_phys=forcing(cfg, cfg.n_coarse))


def snapshot_pair(cfg: KolmogorovConfig, fine: ns.Solver, coarse: ns.Solver):
    """(coarse vorticity, closure target) in physical space for the current
    fine state; ``coarse`` is used as a workspace (its state is overwritten)."""
    wf = fine.get_state_spectral()
    nf = fine.eval_rhs()
    wc = restrict_2d(wf, cfg.n_fine, cfg.n_coarse)
    coarse.set_state_spectral(wc)
    ncoarse = coarse.eval_rhs()
    x = coarse.get_state()
    coarse.set_state_spectral(restrict_2d(nf, cfg.n_fine, cfg.n_coarse) - ncoarse)
    t = coarse.get_state()
    return x, t, wc


def generate(cfg: KolmogorovConfig, seeds, log=None):
    """Snapshots of fine runs (one per seed) filtered to the coarse grid:
    arrays X, T of shape (len(seeds) * snaps_per_seed, N_c, N_c), float32."""
    xs, ts, energy = [], [], []
    with fine_solver(cfg) as fine, coarse_solver(cfg) as coarse:
        for seed in seeds:
            fine.set_state_spectral(inputs.random_vorticity_2d(cfg.n_fine, seed, k0=cfg.ic_k0,
                                                               energy=cfg.ic_energy))
            fine.step(cfg.steps(cfg.t_spin, True))
            for _ in range(cfg.snaps_per_seed):
                fine.step(cfg.steps(cfg.snap_every, True))
                x, t, _ = snapshot_pair(cfg, fine, coarse)
                xs.append(x.astype(np.float32))
                ts.append(t.astype(np.float32))
            energy.append(fine.diagnostics())
            if log:
                log(f"seed {seed}: E, Omega at the last snapshot = {energy[-1]}")
    return np.stack(xs), np.stack(ts), energy


@dataclass
class Trained:
    net: ns.CNN
    x_scale: float
    t_scale: float
    losses: list = field(default_factory=list)


def train(X: np.ndarray, T: np.ndarray, steps: int = 3000, batch: int = 16, lr: float = 1e-3, seed: int = 0,
          log=None, noise: float = 0.0) -> Trained:
    """Adam on the mean squared error of normalised targets; the normalised
    snapshots are uploaded once and each minibatch is gathered on the device,
    on the stream the CNN runs on, from a per-epoch host permutation; cosine
    learning-rate decay.  ``noise`` > 0 adds Gaussian noise of that standard
    deviation to the normalised inputs of every minibatch (the network then
    also sees states perturbed the way its own errors perturb a closed run)."""
    import torch

    n, h, w = X.shape
    x_scale, t_scale = float(X.std()), float(T.std())
    rng = np.random.default_rng(seed)
    net = ns.CNN(h, w, batch, seed=seed)
    losses = []
    per_epoch = n // batch
    xs = torch.from_numpy(np.ascontiguousarray(X / x_scale, dtype=np.float32)).cuda()
    ts = torch.from_numpy(np.ascontiguousarray(T / t_scale, dtype=np.float32)).cuda()
    xb = torch.empty((batch, h, w), dtype=torch.float32, device="cuda")
    tb = torch.empty_like(xb)
    perm = None
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    for k in range(steps):
        e = k % per_epoch
        if e == 0:
            perm = rng.permutation(n)
        idx = torch.from_numpy(perm[e * batch:(e + 1) * batch]).cuda()
        torch.index_select(xs, 0, idx, out=xb)
        torch.index_select(ts, 0, idx, out=tb)
        if noise > 0:
            xb.add_(torch.randn(xb.shape, generator=gen, device="cuda"), alpha=noise)
        lr_k = lr * 0.5 * (1.0 + math.cos(math.pi * k / steps))
        want = (k % 50 == 0) or k == steps - 1
        loss = net.train_step(xb.data_ptr(), tb.data_ptr(), batch, lr_k, want_loss=want,
                              stream=torch.cuda.current_stream().cuda_stream)
        if want:
            losses.append((k, loss))
            if log and k % 500 == 0:
                log(f"step {k}: loss {loss:.4f}")
    torch.cuda.synchronize()
    return Trained(net, x_scale, t_scale, losses)


def predict(tr: Trained, X: np.ndarray) -> np.ndarray:
    """Network prediction of the (unnormalised) closure target for X (B, h, w)."""
    import torch

    out = np.empty_like(X, dtype=np.float32)
    b = tr.net.max_batch
    for i in range(0, X.shape[0], b):
        xb = torch.from_numpy(np.ascontiguousarray(X[i:i + b] / tr.x_scale, dtype=np.float32)).cuda()
        yb = torch.empty_like(xb)
        tr.net.forward(xb.data_ptr(), yb.data_ptr(), xb.shape[0])
        torch.cuda.synchronize()
        out[i:i + b] = yb.cpu().numpy() * tr.t_scale
    return out


def a_priori(tr: Trained, X: np.ndarray, T: np.ndarray) -> dict:
    """Skill of the prediction against the target: the plain coarse solve
    predicts tau = 0, so its mean squared error is mean(tau^2)."""
    P = predict(tr, X).astype(np.float64)
    T = T.astype(np.float64)
    mse = float(np.mean((P - T) ** 2))
    mse0 = float(np.mean(T ** 2))
    corr = float(np.sum(P * T) / math.sqrt(np.sum(P * P) * np.sum(T * T)))
    return {"mse_closure": mse, "mse_plain": mse0, "skill": 1.0 - mse / mse0, "correlation": corr}


class ClosureSolver:
    """Coarse 2D solve with the network's prediction added to the forcing
    before every step; all work enqueued on one CUDA stream.  With
    ``use_graph`` one corrected step (state to physical space, network,
    forcing update, RK4 step) is captured once into a CUDA graph and
    replayed."""

    def __init__(self, cfg: KolmogorovConfig, tr: Trained, check_every: int = 50, blowup: float = 100.0,
                 use_graph: bool = True, fallback: str = "fine"):
        import torch

        if fallback not in ("fine", "coarse"):
            raise ValueError("fallback must be 'fine' or 'coarse'")
        self.fallback = fallback
        self.fine = None  # the plain fine-grid solve, created on fallback
        self.cfg, self.tr = cfg, tr
        n = cfg.n_coarse
        self.n2 = n * n
        self.solver = ns.Solver(2, n, FP32, nu=cfg.nu, dt=cfg.dt_coarse)
        self.stream = torch.cuda.Stream()
        self.solver.set_stream(self.stream.cuda_stream)
        self.F = torch.from_numpy(forcing(cfg, n)).cuda()
        self.phys = torch.empty((n, n), dtype=torch.float64, device="cuda")
        self.f = torch.empty((n, n), dtype=torch.float64, device="cuda")
        self.x = torch.empty((1, n, n), dtype=torch.float32, device="cuda")
        self.y = torch.empty((1, n, n), dtype=torch.float32, device="cuda")
        self.check_every, self.blowup = check_every, blowup
        self.fell_back = False
        self._good = None
        self._omega0 = None
        self.use_graph = use_graph
        self._graph = None

    def close(self):
        self.solver.close()
        if self.fine is not None:
            self.fine.close()
            self.fine = None

    @property
    def on_fine(self) -> bool:
        """True once the run has handed over to the plain fine-grid solve."""
        return self.fine is not None

    def set_state_spectral(self, spec):
        if self.fine is not None:
            self.fine.close()
            self.fine = None
        self._plain_forcing()
        self.solver.set_state_spectral(spec)
        self.stream.synchronize()
        self._good = np.array(spec, copy=True)
        self._omega0 = self.solver.diagnostics()[1]
        self.fell_back = False

    def _coarse_view(self):
        """The coarse workspace holding the current coarse view of the run:
        after a hand-over to the fine grid, the fine state filtered to the
        coarse modes."""
        if self.fine is not None:
            self.solver.set_state_spectral(
                restrict_2d(self.fine.get_state_spectral(), self.cfg.n_fine, self.cfg.n_coarse))
        return self.solver

    def get_state_spectral(self):
        return self._coarse_view().get_state_spectral()

    def diagnostics(self):
        return self._coarse_view().diagnostics()

    def energy_spectrum(self):
        return self._coarse_view().energy_spectrum()

    def _correct(self):
        s, st = self.solver.state, self.stream.cuda_stream
        ns._check(ns.lib.ns_state_to_phys_device(s, ns.ctypes.c_void_p(self.phys.data_ptr())), s)
        ns.f64_to_f32(self.phys.data_ptr(), self.x.data_ptr(), self.n2, 1.0 / self.tr.x_scale, st)
        self.tr.net.forward(self.x.data_ptr(), self.y.data_ptr(), 1, st)
        ns.f32_axpy_f64(self.y.data_ptr(), self.F.data_ptr(), self.f.data_ptr(), self.n2, self.tr.t_scale, st)
        ns._check(ns.lib.ns_set_forcing_phys_device(s, ns.ctypes.c_void_p(self.f.data_ptr())), s)

    def _corrected_step(self):
        self._correct()
        self.solver.step(1)

    def _capture(self):
        """Record one corrected step into a CUDA graph (after an eager step
        has done every lazy set-up: kernel attributes, the step graph)."""
        import torch

        self._corrected_step()
        self.stream.synchronize()
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        self.solver.set_stream(cap.cuda_stream)
        saved = self.stream
        self.stream = cap
        try:
            with torch.cuda.graph(g, stream=cap, capture_error_mode="thread_local"):
                self._corrected_step()
        finally:
            self.stream = saved
            self.solver.set_stream(saved.cuda_stream)
        self._graph = g

    def _run_corrected(self, n: int):
        import torch

        if not self.use_graph:
            for _ in range(n):
                self._corrected_step()
            return
        if self._graph is None:
            self._capture()
            n -= 1  # the eager warm-up step of the capture advanced the state
        with torch.cuda.stream(self.stream):
            for _ in range(n):
                self._graph.replay()

    def _plain_forcing(self):
        s = self.solver.state
        ns._check(ns.lib.ns_set_forcing_phys_device(s, ns.ctypes.c_void_p(self.F.data_ptr())), s)

    def step(self, nsteps: int):
        """Advance by nsteps coarse steps (after a hand-over to the fine grid:
        the same time in fine steps)."""
        if self.fine is not None:
            self.fine.step(nsteps * self.cfg.ratio)
            return
        done = 0
        while done < nsteps:
            chunk = min(self.check_every, nsteps - done)
            if self.fine is not None:
                self.fine.step(chunk * self.cfg.ratio)
            elif self.fell_back:
                self.solver.step(chunk)
            else:
                self._run_corrected(chunk)
            done += chunk
            if not self.fell_back:
                try:
                    om = self.solver.diagnostics()[1]
                    ok = math.isfinite(om) and om <= self.blowup * self._omega0
                except ns.NSError:
                    ok = False
                if ok:
                    self._good = self.solver.get_state_spectral()
                else:
                    self.fell_back = True
                    self._plain_forcing()
                    self.solver.set_state_spectral(self._good)
                    if self.fallback == "fine":
                        self.fine = fine_solver(self.cfg)
                        self.fine.set_state_spectral(prolong_2d(self._good, self.cfg.n_coarse, self.cfg.n_fine))


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    w = np.where(np.arange(b.shape[-1]) == 0, 1.0, 2.0)
    return float(np.sqrt(np.sum(w * np.abs(a - b) ** 2) / np.sum(w * np.abs(b) ** 2)))


def a_posteriori(cfg: KolmogorovConfig, tr: Trained, seed: int, t_eval: float, every: float, log=None) -> dict:
    """From the filtered fine state after spin-up, run the plain coarse solve
    and the closed coarse solve beside the fine solve; at each checkpoint
    compare both with the filtered fine state: vorticity error, enstrophy,
    and the shell energy spectrum (mean |log ratio| over shells 1..kc).  The
    library's own diagnostics evaluate all three states (the filtered fine
    one through a coarse workspace state)."""
    nc = cfg.n_coarse
    kc = inputs.truncation(nc)[0]
    sh = slice(1, kc + 1)
    rows = []
    with fine_solver(cfg) as fine, coarse_solver(cfg) as plain, coarse_solver(cfg) as filtered:
        closed = ClosureSolver(cfg, tr)
        try:
            fine.set_state_spectral(inputs.random_vorticity_2d(cfg.n_fine, seed, k0=cfg.ic_k0, energy=cfg.ic_energy))
            fine.step(cfg.steps(cfg.t_spin, True))
            w0 = restrict_2d(fine.get_state_spectral(), cfg.n_fine, nc)
            plain.set_state_spectral(w0)
            closed.set_state_spectral(w0)
            t = 0.0
            for _ in range(int(round(t_eval / every))):
                fine.step(cfg.steps(every, True))
                plain.step(cfg.steps(every, False))
                closed.step(cfg.steps(every, False))
                t += every
                ref = restrict_2d(fine.get_state_spectral(), cfg.n_fine, nc)
                filtered.set_state_spectral(ref)
                wp, wq = plain.get_state_spectral(), closed.get_state_spectral()
                er, ep, eq = filtered.energy_spectrum(), plain.energy_spectrum(), closed.energy_spectrum()

                def spec_err(e):
                    return float(np.mean(np.abs(np.log(np.maximum(e[sh], 1e-300) / np.maximum(er[sh], 1e-300)))))

                row = {"t": round(t, 6), "err_plain": rel_l2(wp, ref), "err_closure": rel_l2(wq, ref),
                       "enstrophy_fine": filtered.diagnostics()[1], "enstrophy_plain": plain.diagnostics()[1],
                       "enstrophy_closure": closed.diagnostics()[1],
                       "spec_err_plain": spec_err(ep), "spec_err_closure": spec_err(eq),
                       "fell_back": closed.fell_back, "on_fine": closed.on_fine}
                rows.append(row)
                if log:
                    log(json.dumps(row))
        finally:
            closed.close()
    return {"rows": rows}


def step_times(cfg: KolmogorovConfig, tr: Trained, nsteps: int = 200) -> dict:
    """Wall time per step of the plain coarse, closed coarse and fine solves
    (after warm-up, synchronised)."""
    import torch

    out = {}
    w = inputs.random_vorticity_2d(cfg.n_coarse, 1, k0=cfg.ic_k0, energy=cfg.ic_energy)
    wf = inputs.random_vorticity_2d(cfg.n_fine, 1, k0=cfg.ic_k0, energy=cfg.ic_energy)
    with coarse_solver(cfg) as plain, fine_solver(cfg) as fine:
        closed = ClosureSolver(cfg, tr, check_every=10 ** 9)
        eager = ClosureSolver(cfg, tr, check_every=10 ** 9, use_graph=False)
        try:
            for name, s, init in (("plain_coarse", plain, w), ("closure_coarse", closed, w),
                                  ("closure_coarse_eager", eager, w), ("fine", fine, wf)):
                s.set_state_spectral(init)
                s.step(10)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                s.step(nsteps)
                if isinstance(s, ClosureSolver):
                    s.stream.synchronize()
                else:
                    s.sync()
                torch.cuda.synchronize()
                out[name + "_ms"] = 1e3 * (time.perf_counter() - t0) / nsteps
        finally:
            closed.close()
            eager.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description="Train and evaluate the learned closure on forced Kolmogorov flow")
    ap.add_argument("--n-fine", type=int, default=2048)
    ap.add_argument("--n-coarse", type=int, default=256)
    ap.add_argument("--seeds", type=int, default=16)
    ap.add_argument("--snaps", type=int, default=125)
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--noise", type=float, default=0.0, help="input noise (std, normalised units) in training")
    ap.add_argument("--t-eval", type=float, default=2.0)
    ap.add_argument("--every", type=float, default=0.25)
    ap.add_argument("--out", default=None)
    ap.add_argument("--data", default=None, help="npz file: the generated snapshots are loaded from it if it "
                    "exists, else saved to it (several trainings on one data set)")
    a = ap.parse_args(argv)
    cfg = KolmogorovConfig(n_fine=a.n_fine, n_coarse=a.n_coarse, snaps_per_seed=a.snaps,
                           train_seeds=tuple(range(a.seeds)))

    def log(m):
        print(m, flush=True)

    t0 = time.perf_counter()
    if a.data and os.path.exists(a.data):
        d = np.load(a.data)
        X, T, energy = d["X"], d["T"], [tuple(e) for e in d["energy"]]
    else:
        X, T, energy = generate(cfg, cfg.train_seeds, log)
        if a.data:
            np.savez(a.data, X=X, T=T, energy=np.array(energy))
    t_gen = time.perf_counter() - t0
    log(f"generated {X.shape[0]} snapshots in {t_gen:.1f} s; std(omega_c) {X.std():.3f} std(tau) {T.std():.4f}")
    t0 = time.perf_counter()
    tr = train(X, T, steps=a.train_steps, batch=a.batch, lr=a.lr, log=log, noise=a.noise)
    t_train = time.perf_counter() - t0
    Xe, Te, _ = generate(KolmogorovConfig(**{**asdict(cfg), "snaps_per_seed": 20}), (cfg.eval_seed,))
    prior = a_priori(tr, Xe, Te)
    log("a priori (seed %d): %s" % (cfg.eval_seed, json.dumps(prior)))
    post = a_posteriori(cfg, tr, cfg.eval_seed, a.t_eval, a.every, log)
    times = step_times(cfg, tr)
    result = {"config": {k: (list(v) if isinstance(v, tuple) else v) for k, v in asdict(cfg).items()},
              "train": {"steps": a.train_steps, "batch": a.batch, "lr": a.lr, "noise": a.noise,
                        "snapshots": int(X.shape[0]),
                        "gen_s": t_gen, "train_s": t_train, "loss_first": tr.losses[0][1],
                        "loss_last": tr.losses[-1][1]},
              "fine_energy_enstrophy_last": energy, "a_priori": prior, "a_posteriori": post["rows"],
              "step_ms": times}
    if a.out:
        with open(a.out, "w") as f:
            json.dump(result, f, indent=1)
    log(json.dumps({k: result[k] for k in ("a_priori", "step_ms")}))
    tr.net.close()
    return result


if __name__ == "__main__":
    main()
