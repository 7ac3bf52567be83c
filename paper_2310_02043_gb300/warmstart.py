"""Surrogate warm start for lighting optimisation.

The irradiance surrogate (``surrogate.Surrogate``) is fitted to the light
tracer's own irradiance for many single spots, then minimises the design
objective (Eq. 6) cheaply and without Monte Carlo noise; the tracer takes over
from the surrogate's optimum (adjoint light tracing, Alg. 2) and judges every
result. ``SurrogateProblem`` has the interface of ``optim.LightingProblem``,
so the optimisers of ``optim`` drive either.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import optim, scenes
from .surrogate import Surrogate


def _host(x):
    """numpy view of a host array or a torch tensor (copied off the device)."""
    if isinstance(x, torch.Tensor):
        return x.detach().cpu().numpy()
    return np.asarray(x)


def texel_inputs(tracer):
    """Texel centres, normals and areas of the tracer's scene, and the
    normalised box (lo, ext) with a 1 % margin."""
    pos, nrm = tracer.texel_centres()
    area = tracer.texel_areas()
    lo_b, hi_b = pos.min(0), pos.max(0)
    ext = float((hi_b - lo_b).max()) * 1.02
    lo = (lo_b - 0.01 * ext).astype(np.float32)
    return pos, nrm, np.asarray(area, np.float32), lo, ext


def generate_solves(tracer, lights, photons: int, hits: int, seed: int = 0):
    """Irradiance of every light alone, traced with `photons` photons:
    a CUDA tensor [len(lights), n_texels]."""
    n = tracer.n_texels
    E = torch.empty((lights.shape[0], n), dtype=torch.float32, device="cuda")
    for s in range(lights.shape[0]):
        tracer.set_lights(lights[s:s + 1])
        tracer.trace_forward(seed + 7919 * s, photons, hits)
        tracer.irradiance(out=E[s])
    torch.cuda.synchronize()
    return E


def train(sg: Surrogate, steps: int, batch: int = 1 << 18, lr: float = 1e-2, lr_end: float = 1e-3, seed: int = 0,
          callback=None):
    """Adam steps on random (solve, texel) batches with an exponentially
    decaying learning rate; returns the batch losses."""
    losses = []
    for k in range(steps):
        rate = lr * (lr_end / lr) ** (k / max(1, steps - 1))
        losses.append(sg.train_step(seed, batch, rate))
        if callback is not None:
            callback(k, losses[-1])
    return losses


def fit(tracer, n_solves: int = 4096, photons: int = 1 << 20, hits: int = 5, steps: int = 2000,
        batch: int = 1 << 18, lr: float = 1e-2, lr_end: float = 1e-3, seed: int = 0, device: int = 0):
    """Train a surrogate on the tracer's scene: n_solves single-spot solves
    (``scenes.surrogate_training_lights``), then `steps` Adam steps. Returns
    (surrogate, info) with timings and losses."""
    info = {}
    t0 = time.perf_counter()
    lights = scenes.surrogate_training_lights(seed, n_solves)
    E = generate_solves(tracer, lights, photons, hits, seed)
    info["solve_s"] = time.perf_counter() - t0
    sg = Surrogate(device)
    pos, nrm, area, lo, ext = texel_inputs(tracer)
    sg.set_texels(pos, nrm, area, lo, ext)
    W, table = scenes.surrogate_init(seed)
    sg.set_params(W, table)
    sg.set_training_data(lights, E)
    sg._solves = E
    t1 = time.perf_counter()
    info["losses"] = train(sg, steps, batch, lr, lr_end, seed)
    torch.cuda.synchronize()
    info["train_s"] = time.perf_counter() - t1
    return sg, info


class SurrogateProblem:
    """The design objective evaluated by the surrogate: forward_loss returns
    O and keeps dO/dp, which adjoint returns (one sg_design call computes
    both; the seeds are unused, the objective is deterministic)."""

    def __init__(self, sg: Surrogate, target, alpha=None):
        self.sg = sg
        self.target = torch.as_tensor(_host(target).astype(np.float32), device="cuda")
        self.alpha = None if alpha is None else torch.as_tensor(_host(alpha).astype(np.float32), device="cuda")
        self._token = 0
        self._grad = None
        self.evaluations = 0

    def forward_loss(self, lights, seed: int = 0):
        O, g = self.sg.design(lights, self.target, self.alpha)
        self._token += 1
        self._grad = g
        self.evaluations += 1
        return O, self._token

    def adjoint(self, lights, seed_fwd: int, seed_adj: int, token: int):
        if token != self._token:
            self.forward_loss(lights)
        return self._grad

    def objective(self, rig, seed_fwd: int = 0, seed_adj: int = 0):
        return optim.TraceObjective.apply(rig.physical(), rig.types, self, seed_fwd, seed_adj)


def relative_loss(tracer, lights, target, area, photons: int, hits: int, seed: int, alpha=None) -> float:
    """Noise-free estimate of the relative objective O / (1/2 sum A alpha E*^2):
    with two independent traces E1, E2 of the same lights, 1/2 sum A alpha
    (E1 - E*)(E2 - E*) has the expectation of the objective of the mean
    irradiance (the Monte Carlo variance cancels)."""
    tracer.set_lights(lights)
    tracer.trace_forward(seed, photons, hits)
    E1 = tracer.irradiance().astype(np.float64)
    tracer.trace_forward(seed + 1, photons, hits)
    E2 = tracer.irradiance().astype(np.float64)
    t = _host(target).astype(np.float64)
    a = np.ones_like(t) if alpha is None else _host(alpha).astype(np.float64)
    A = np.asarray(area, np.float64)
    return float(np.sum(A * a * (E1 - t) * (E2 - t)) / np.sum(A * a * t * t))


def time_to_loss(tracer, scene, start, target, phases, threshold: float, area, eval_photons: int = 1 << 24,
                 hits: int = 5, eval_every: int = 10, max_seconds: float = 60.0,
                 optimize=("x", "y", "yaw", "pitch", "p_int", "theta_in")):
    """Runs the optimisation phases in order -- ("surrogate", problem, steps,
    lr) or ("tracer", photons, steps, lr) -- with Adam from `start`, and every
    `eval_every` steps measures the noise-free relative loss with the tracer
    (untimed). Returns (seconds of optimisation until the loss first reached
    `threshold` or None, history [(phase, step, seconds, relative loss)])."""
    rig = optim.LightRig(start, optimize=optimize)
    target = _host(target).astype(np.float32)
    timed, hist, reached = 0.0, [], None
    for phase in phases:
        kind, steps, lr = phase[0], phase[2], phase[3]
        if kind == "surrogate":
            prob, sched = phase[1], optim.SeedSchedule(base=1, fixed=True)
        else:
            prob = optim.LightingProblem(scene, target, photons=phase[1], hits=hits, tracer=tracer)
            sched = optim.SeedSchedule(base=11)
        opt = torch.optim.Adam([rig.params], lr=lr, betas=(0.9, 0.999))
        for k in range(steps):
            torch.cuda.synchronize()
            a = time.perf_counter()
            optim.adam(prob, rig, 1, lr, sched, start_step=k, optimizer=opt)
            torch.cuda.synchronize()
            timed += time.perf_counter() - a
            if (k + 1) % eval_every == 0 or k == steps - 1:
                r = relative_loss(tracer, rig.lights(), target, area, eval_photons, hits, 100003 + len(hist))
                hist.append((kind, k + 1, timed, r))
                if reached is None and r <= threshold:
                    reached = timed
                    return reached, hist, rig.lights()
                if timed > max_seconds:
                    return reached, hist, rig.lights()
    return reached, hist, rig.lights()

