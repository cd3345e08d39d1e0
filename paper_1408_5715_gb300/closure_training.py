"""Training and evaluation of the learned dissipation scale (not in the paper).

Data: the channel with the circular-arc bump at a coarse resolution, and the
same channel refined twice by edge midpoints (16 fine triangles per coarse
one).  For each inflow Mach number the fine mesh is run by the FP64 path of
this library from the uniform free stream; snapshots of the fine state are
restricted to the coarse cells (area-weighted means of the 16 children).
Each training sample is a pair (R U_f(t), R U_f(t + dt_c)): one coarse
forward-Euler step of size dt_c with the closure, started from the first
state, should reproduce the second.  The loss, its gradient and the Adam
update run in the library's kernels (fv_closure_loss_grad, fv_adam_step);
this module only moves tensors between them.

Evaluation: on held-out Mach numbers, the coarse mesh is run from the free
stream to the horizon T with plain Lax-Friedrichs and with the closure; both
are compared with the restricted fine FP64 solution (relative L2 error of the
density, area weighted).
"""
from __future__ import annotations

import math
import time
from dataclasses import asdict, dataclass, field

import numpy as np

from . import binding as B
from . import workloads as W


@dataclass
class TrainConfig:
    coarse_nx: int = 250
    coarse_ny: int = 80
    levels: int = 2
    n_train: int = 16
    n_test: int = 4
    mach_lo: float = 0.4
    mach_hi: float = 0.7
    horizon: float = 0.6
    pairs_per_run: int = 40
    epochs: int = 40
    lr: float = 2e-3
    init_scale: float = 0.05
    seed: int = 5
    info: dict = field(default_factory=dict)


def logit(p):
    return math.log(p / (1.0 - p))


def initial_theta(seed, scale):
    """Small random weights with s = 1 (the plain flux) at zero input."""
    rng = np.random.default_rng(seed)
    th = (rng.normal(size=B.CLOSURE_PARAMS) * scale).astype(np.float32)
    th[-33:-1] = 0.0  # w3: start exactly at the plain flux
    th[-1] = logit(0.8 / 1.3)
    return th


class Problem:
    """Coarse and fine meshes, restriction, and the fixed coarse time step."""

    def __init__(self, cfg: TrainConfig):
        import torch
        self.cfg = cfg
        self.mi_c = W.channel_bump(cfg.coarse_nx, cfg.coarse_ny, seed=cfg.seed)
        self.mi_f, parent = W.refine_midpoint(self.mi_c, cfg.levels)
        self.kids = 4 ** cfg.levels
        self.mc = B.Mesh.from_input(self.mi_c, "f32")
        self.mf = B.Mesh.from_input(self.mi_f, "f64")
        # Hilbert order: compact warps share MLP rows (coarse) and compact
        # tiles serve the shared-memory shape (fine); the fine shape is tuned
        self.perm_c = self.mc.renumber("hilbert")
        self.perm_f = self.mf.renumber("hilbert")
        U = torch.tensor(W.uniform_state(self.mf.n, W.freestream(0.5)), dtype=torch.float64,
                         device="cuda")
        self.fine_shape, _ = self.mf.autotune(U)
        del U
        _, _, self.area_c = self.mc.export()  # coarse areas, coarse numbering
        _, _, area_f = self.mf.export()
        self.n_c, self.n_f = self.mc.n, self.mf.n
        # the children of coarse cell i (coarse numbering) are fine cells
        # perm_c[i] * kids + j of the refinement order; in the fine numbering
        inv_f = np.empty(self.n_f, np.int64)
        inv_f[self.perm_f] = np.arange(self.n_f)
        kids_of = inv_f[self.perm_c[:, None] * self.kids + np.arange(self.kids)[None, :]]
        self.fine_of = torch.tensor(kids_of.astype(np.int32), device="cuda")
        self.area_f = torch.tensor(area_f, dtype=torch.float64, device="cuda")

    def restrict(self, Uf):
        """Fine FP64 state (fine numbering) -> coarse FP32 state (coarse
        numbering): area-weighted means of the children (fv_restrict_mean)."""
        import torch
        Uc = torch.empty((self.n_c, 4), dtype=torch.float32, device="cuda")
        return B.restrict_mean(Uf, self.area_f, self.fine_of, Uc)

    def set_mach(self, mach):
        prim = W.freestream(mach)
        self.mc.set_freestream(*prim)
        self.mf.set_freestream(*prim)
        return prim

    def coarse_dt(self, machs):
        """One fixed coarse step for all runs: 0.3 of the CFL bound of the
        fastest free stream (the flow speeds up over the bump)."""
        import torch
        dts = []
        for m in machs:
            prim = self.set_mach(m)
            U = torch.tensor(W.uniform_state(self.n_c, prim), dtype=torch.float32, device="cuda")
            dts.append(self.mc.compute_dt(U, 0.3))
        return min(dts)


def advance(mesh, U, duration, cfl=0.4):
    """Advances U by exactly ``duration`` with CFL time steps (the last one
    clamped).  Steps are requested in batches sized from the current dt, so
    that few steps past the target are launched (they advance nothing)."""
    done = 0.0
    while duration - done > 1e-15 * max(duration, 1.0):
        dt = mesh.compute_dt(U, cfl)
        n = int(math.ceil((duration - done) / (0.9 * dt))) + 2
        done += mesh.step(U, n, cfl, t_stop=duration - done)
    return done


def fine_pairs(prob: Problem, mach, dt_c, horizon, n_pairs):
    """Restricted fine snapshot pairs (t, t + dt_c) spread over [0, horizon),
    and the restricted fine state at the horizon."""
    import torch
    prim = prob.set_mach(mach)
    Uf = torch.tensor(W.uniform_state(prob.n_f, prim), dtype=torch.float64, device="cuda")
    starts = np.linspace(0.0, horizon - dt_c, n_pairs + 1)[1:]
    t = 0.0
    pairs = []
    for ts in starts:
        if ts > t:
            t += advance(prob.mf, Uf, ts - t)
        a = prob.restrict(Uf)
        t += advance(prob.mf, Uf, dt_c)
        pairs.append((a, prob.restrict(Uf)))
    if horizon > t:
        t += advance(prob.mf, Uf, horizon - t)
    return pairs, prob.restrict(Uf)


def rel_l2_rho(prob: Problem, Uc, ref):
    """Area-weighted relative L2 error of the density, on the host."""
    v = prob.area_c
    a = Uc[:, 0].double().cpu().numpy()
    b = ref[:, 0].double().cpu().numpy()
    return float(np.sqrt((v * (a - b) ** 2).sum() / (v * b * b).sum()))


def coarse_run(prob: Problem, mach, dt_c, horizon, closure=None):
    import torch
    prim = prob.set_mach(mach)
    U = torch.tensor(W.uniform_state(prob.n_c, prim), dtype=torch.float32, device="cuda")
    nsteps = int(round(horizon / dt_c))
    prob.mc.step(U, nsteps, -dt_c, closure=closure)
    return U, nsteps


def train_and_evaluate(cfg: TrainConfig = TrainConfig(), log=None):
    """Runs the whole pipeline; returns a report dict."""
    import torch
    t_start = time.perf_counter()
    rng = np.random.default_rng(cfg.seed)
    machs = rng.uniform(cfg.mach_lo, cfg.mach_hi, size=cfg.n_train + cfg.n_test)
    train_m, test_m = machs[:cfg.n_train], machs[cfg.n_train:]
    prob = Problem(cfg)
    dt_c = prob.coarse_dt(list(machs))
    # ---- data
    t0 = time.perf_counter()
    samples = []  # (mach, U0, Ut)
    for m in train_m:
        pairs, _ = fine_pairs(prob, m, dt_c, cfg.horizon, cfg.pairs_per_run)
        samples += [(m, a, b) for a, b in pairs]
    refs = {}
    for m in test_m:
        _, refs[m] = fine_pairs(prob, m, dt_c, cfg.horizon, 1)
    t_data = time.perf_counter() - t0
    # loss weights: RMS one-step change of each conserved component
    inc = torch.stack([(b - a).double().pow(2).mean(dim=0) for _, a, b in samples]).mean(dim=0)
    w = tuple(float(x) for x in torch.sqrt(inc).clamp_min(1e-12))
    # ---- training
    theta = torch.tensor(initial_theta(cfg.seed, cfg.init_scale), device="cuda")
    mom1, mom2 = torch.zeros_like(theta), torch.zeros_like(theta)
    cl = B.Closure(theta.cpu().numpy())
    grad = torch.empty_like(theta)

    def epoch_loss():
        tot = 0.0
        for m, a, b in samples:
            prob.set_mach(m)
            tot += cl.loss_grad(prob.mc, a, b, dt_c, w, grad=grad)[0]
        return tot / len(samples)

    loss0 = epoch_loss()
    step = 0
    t0 = time.perf_counter()
    history = [loss0]
    for ep in range(cfg.epochs):
        order = rng.permutation(len(samples))
        for k in order:
            m, a, b = samples[k]
            prob.set_mach(m)
            cl.loss_grad(prob.mc, a, b, dt_c, w, grad=grad)
            step += 1
            B.adam_step(theta, grad, mom1, mom2, step, lr=cfg.lr)
            cl.set(theta)
        if ep % 10 == 9 or ep == cfg.epochs - 1:
            history.append(epoch_loss())
            if log:
                log(f"epoch {ep + 1}: mean one-step loss {history[-1]:.4g}")
    t_train = time.perf_counter() - t0
    # ---- held-out evaluation against the restricted fine solution
    res = []
    for m in test_m:
        Up, nsteps = coarse_run(prob, m, dt_c, cfg.horizon)
        Ul, _ = coarse_run(prob, m, dt_c, cfg.horizon, closure=cl)
        res.append({"mach": float(m), "steps": nsteps,
                    "err_plain": rel_l2_rho(prob, Up, refs[m]),
                    "err_learned": rel_l2_rho(prob, Ul, refs[m])})
    scales = cl.scales(prob.mc, Ul).cpu().numpy()
    report = {
        "config": asdict(cfg), "coarse_cells": prob.n_c, "fine_cells": prob.n_f,
        "fine_kernel_shape": prob.fine_shape,
        "dt_coarse": dt_c, "train_machs": [float(x) for x in train_m],
        "test_machs": [float(x) for x in test_m], "samples": len(samples),
        "loss_weights": w, "loss_first": loss0, "loss_history": history,
        "heldout": res,
        "mean_err_plain": float(np.mean([r["err_plain"] for r in res])),
        "mean_err_learned": float(np.mean([r["err_learned"] for r in res])),
        "scale_stats": {"min": float(scales.min()), "mean": float(scales.mean()),
                        "max": float(scales.max())},
        "seconds": {"fine_data": t_data, "training": t_train,
                    "total": time.perf_counter() - t_start},
        "theta": theta.cpu().numpy(),
    }
    return report, cl, prob


def step_cost(prob_or_mesh, closure, steps=200):
    """Microseconds per forward-Euler step of a coarse mesh with and without
    the closure (CUDA events, fixed dt)."""
    import torch
    mesh = prob_or_mesh.mc if isinstance(prob_or_mesh, Problem) else prob_or_mesh
    U0 = torch.tensor(W.uniform_state(mesh.n, W.freestream(0.5)), dtype=torch.float32,
                      device="cuda")
    dt = mesh.compute_dt(U0, 0.3)
    out = {}
    for name, cl in (("plain", None), ("learned", closure)):
        U = U0.clone()
        mesh.step(U, 20, -dt, closure=cl)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mesh.step(U, steps, -dt, closure=cl, sync=False)
        e1.record()
        torch.cuda.synchronize()
        out[name] = 1e3 * e0.elapsed_time(e1) / steps
    return out


def main(argv=None):
    import argparse
    import json
    import torch
    p = argparse.ArgumentParser(description="train and evaluate the learned dissipation scale")
    p.add_argument("--coarse-nx", type=int, default=TrainConfig.coarse_nx)
    p.add_argument("--coarse-ny", type=int, default=TrainConfig.coarse_ny)
    p.add_argument("--n-train", type=int, default=TrainConfig.n_train)
    p.add_argument("--n-test", type=int, default=TrainConfig.n_test)
    p.add_argument("--horizon", type=float, default=TrainConfig.horizon)
    p.add_argument("--pairs", type=int, default=TrainConfig.pairs_per_run)
    p.add_argument("--epochs", type=int, default=TrainConfig.epochs)
    p.add_argument("--lr", type=float, default=TrainConfig.lr)
    p.add_argument("--seed", type=int, default=TrainConfig.seed)
    a = p.parse_args(argv)
    torch.cuda.set_device(0)
    cfg = TrainConfig(coarse_nx=a.coarse_nx, coarse_ny=a.coarse_ny, n_train=a.n_train,
                      n_test=a.n_test, horizon=a.horizon, pairs_per_run=a.pairs,
                      epochs=a.epochs, lr=a.lr, seed=a.seed)
    report, cl, prob = train_and_evaluate(cfg, log=lambda m: print(m, flush=True))
    report["step_cost_us"] = step_cost(prob, cl)
    report.pop("theta")
    print(json.dumps(report), flush=True)


if __name__ == "__main__":
    main()
