"""Gradient-based lighting optimisation on top of the tracer.

``TraceObjective`` is a ``torch.autograd.Function``: its forward pass traces
photons and evaluates the texel objective (Alg. 1, Eq. 6); its backward pass
replays the same photon paths from their random-number counters and returns
dO/dp (Alg. 2, Eq. 11). Nothing about the paths is stored between the two
passes: the adjoint recomputes them (the paper's per-path adjoint states,
Sec. 4.3); within the adjoint pass each photon leaves a 16-byte record (its
adjoint state and first hit) for the gradient kernel. If another
forward pass ran in between (an L-BFGS line search does this), the backward
pass first re-runs forward and loss for its own parameters.

Optimisers are PyTorch's: Adam with beta = (0.9, 0.999) as in the paper's
results, and L-BFGS with a strong-Wolfe line search on a fixed seed (the
line search needs a deterministic objective; Sec. 4.3's correlated
evaluation).
"""
from __future__ import annotations

import dataclasses
import json
import os
import time

import numpy as np
import torch

PARAM_NAMES = ("x", "y", "z", "yaw", "pitch", "p_int", "theta_in", "theta_out")


class LightRig(torch.nn.Module):
    """Luminaire parameters [L, 8] (float64) with the light types fixed.

    ``optimize`` names the parameter columns that change; the others keep
    their values (their gradients are zeroed). ``scale`` (8 values, default
    ones) sets the unit of each column for the optimiser: ``params`` holds
    the parameters divided by it, so a step of a given size in ``params`` is
    a step of scale times that size in metres or radians (a learning rate in
    scaled units)."""

    def __init__(self, lights, optimize=("x", "y", "z", "yaw", "pitch", "p_int", "theta_in"), scale=None):
        super().__init__()
        arr = np.asarray(lights, np.float64).reshape(-1, 9)
        self.register_buffer("types", torch.tensor(arr[:, 0]))
        sc = torch.ones(8, dtype=torch.float64) if scale is None else torch.tensor(scale, dtype=torch.float64)
        if sc.shape != (8,) or not bool(torch.all(sc > 0)):
            raise ValueError("scale needs 8 positive values")
        self.register_buffer("scale", sc)
        self.params = torch.nn.Parameter(torch.tensor(arr[:, 1:9] / sc.numpy()))
        mask = torch.zeros(8, dtype=torch.bool)
        for name in optimize:
            mask[PARAM_NAMES.index(name)] = True
        self.register_buffer("mask", mask)

    def physical(self) -> torch.Tensor:
        """The parameters in metres / radians / p_int (differentiable)."""
        return self.params * self.scale

    def lights(self) -> np.ndarray:
        """[L, 9] rows (type, x, y, z, yaw, pitch, p_int, theta_in, theta_out)."""
        p = self.physical().detach().cpu().numpy()
        return np.ascontiguousarray(np.concatenate([self.types.cpu().numpy()[:, None], p], axis=1))

    @torch.no_grad()
    def project(self):
        """Keep every spot valid: 0 <= theta_in < theta_out <= pi."""
        p = self.params * self.scale
        p[:, 7].clamp_(1e-3, np.pi)
        p[:, 6].copy_(torch.minimum(p[:, 6].clamp(min=0.0), p[:, 7] - 1e-3))
        self.params.copy_(p / self.scale)

    def mask_grad(self):
        if self.params.grad is not None:
            self.params.grad[:, ~self.mask] = 0.0


@dataclasses.dataclass
class SeedSchedule:
    """Random-number seeds of the forward and adjoint passes per step.

    correlated: the adjoint replays the forward pass's paths (validation, FD);
    otherwise it draws new ones (decorrelated, Sec. 4.3). fixed: every step
    uses the same seeds (a deterministic objective, needed by L-BFGS)."""
    base: int = 1
    correlated: bool = False
    fixed: bool = False

    def seeds(self, step: int):
        s = self.base if self.fixed else self.base + 7919 * step
        return s, (s if self.correlated else s + 1)


class LightingProblem:
    """A scene, its target irradiance and the photon budget, bound to a tracer.

    ``tracer`` is any object with the methods of ``lighttrace.Tracer``; by
    default a new CUDA tracer on ``device``."""

    def __init__(self, scene, target, alpha=None, photons: int = 1 << 20, hits: int = 3, device: int = 0,
                 tracer=None):
        if tracer is None:
            from .lighttrace import Tracer
            tracer = Tracer(device)
        self.tr = tracer
        self.scene = scene
        self.photons = int(photons)
        self.hits = int(hits)
        self.n_texels = self.tr.upload_scene(scene)
        self.tr.set_target(np.ascontiguousarray(target, np.float32),
                           None if alpha is None else np.ascontiguousarray(alpha, np.float32))
        self._token = 0          # identifies the forward pass whose weights the tracer holds
        self.evaluations = 0

    def forward_loss(self, lights, seed: int) -> tuple[float, int]:
        self.tr.set_lights(lights)
        self.tr.trace_forward(seed, self.photons, self.hits)
        O = float(self.tr.loss())
        self._token += 1
        self.evaluations += 1
        return O, self._token

    def adjoint(self, lights, seed_fwd: int, seed_adj: int, token: int) -> np.ndarray:
        if token != self._token:
            self.forward_loss(lights, seed_fwd)      # recompute: the weights belong to another pass
        return np.asarray(self.tr.trace_adjoint(seed_adj, self.photons, self.hits), np.float64)

    def objective(self, rig: LightRig, seed_fwd: int, seed_adj: int) -> torch.Tensor:
        return TraceObjective.apply(rig.physical(), rig.types, self, seed_fwd, seed_adj)


class TraceObjective(torch.autograd.Function):
    """O(p) by light tracing; dO/dp by adjoint light tracing (path replay)."""

    @staticmethod
    def forward(ctx, params, types, problem, seed_fwd, seed_adj):
        lights = np.concatenate([types.detach().cpu().numpy()[:, None], params.detach().cpu().numpy()], axis=1)
        O, token = problem.forward_loss(lights, seed_fwd)
        ctx.problem, ctx.lights, ctx.token = problem, lights, token
        ctx.seed_fwd, ctx.seed_adj = seed_fwd, seed_adj
        ctx.device, ctx.dtype = params.device, params.dtype
        return torch.tensor(O, dtype=params.dtype, device=params.device)

    @staticmethod
    def backward(ctx, grad_out):
        g = ctx.problem.adjoint(ctx.lights, ctx.seed_fwd, ctx.seed_adj, ctx.token)
        grad = torch.from_numpy(g).to(device=ctx.device, dtype=ctx.dtype) * grad_out
        return grad, None, None, None, None


def adam(problem: LightingProblem, rig: LightRig, steps: int, lr: float = 0.05,
         schedule: SeedSchedule | None = None, start_step: int = 0, optimizer=None, callback=None):
    """Adam on the rig's selected parameters; returns (losses, optimizer)."""
    schedule = schedule or SeedSchedule()
    opt = optimizer or torch.optim.Adam([rig.params], lr=lr, betas=(0.9, 0.999))
    losses = []
    for k in range(start_step, start_step + steps):
        sf, sa = schedule.seeds(k)
        opt.zero_grad(set_to_none=False)
        loss = problem.objective(rig, sf, sa)
        loss.backward()
        rig.mask_grad()
        opt.step()
        rig.project()
        losses.append(float(loss.detach()))
        if callback is not None:
            callback(k, losses[-1], rig)
    return losses, opt


def lbfgs(problem: LightingProblem, rig: LightRig, max_iter: int = 20, seed: int = 1, lr: float = 1.0,
          history_size: int = 10):
    """L-BFGS with a strong-Wolfe line search on a fixed seed; returns the
    objective after every evaluation."""
    opt = torch.optim.LBFGS([rig.params], lr=lr, max_iter=max_iter, history_size=history_size,
                            line_search_fn="strong_wolfe")
    trace = []

    def closure():
        opt.zero_grad(set_to_none=False)
        loss = problem.objective(rig, seed, seed)
        loss.backward()
        rig.mask_grad()
        trace.append(float(loss.detach()))
        return loss

    opt.step(closure)
    rig.project()
    return trace


class MetricsLog:
    """Per-iteration metrics of an optimisation run as JSON lines (append
    mode, one object per step, flushed as written): the step, its objective,
    its seeds, the norm of the gradient of every parameter column that
    changes, and the seconds since the log was opened. Pass it as the
    ``callback`` of ``adam``; a run resumed from a checkpoint appends to the
    same file."""

    def __init__(self, path: str, schedule: SeedSchedule | None = None):
        self.path, self.schedule = path, schedule
        self.t0 = time.perf_counter()
        self.f = open(path, "a", buffering=1)

    def __call__(self, step: int, loss: float, rig: LightRig):
        rec = {"step": int(step), "loss": float(loss), "t_s": time.perf_counter() - self.t0}
        if self.schedule is not None:
            rec["seeds"] = list(self.schedule.seeds(step))
        if rig.params.grad is not None:
            g = (rig.params.grad / rig.scale).detach().cpu().numpy()      # dO/dp in physical units
            rec["grad_norm"] = {PARAM_NAMES[j]: float(np.linalg.norm(g[:, j]))
                                for j in range(8) if bool(rig.mask[j])}
        self.f.write(json.dumps(rec) + "\n")

    def close(self):
        self.f.close()


def save_checkpoint(path: str, rig: LightRig, optimizer, step: int, schedule: SeedSchedule):
    """Parameters, optimiser state, step index and seed schedule. The seeds of
    step k depend only on (schedule, k), so a resumed run repeats the same
    random numbers as an uninterrupted one."""
    tmp = path + ".tmp"
    torch.save({"params": rig.params.detach().clone(), "types": rig.types.clone(), "mask": rig.mask.clone(),
                "scale": rig.scale.clone(),
                "optimizer": optimizer.state_dict(), "step": step, "schedule": dataclasses.asdict(schedule)}, tmp)
    os.replace(tmp, path)


def load_checkpoint(path: str, rig: LightRig, optimizer):
    """Restore a checkpoint into rig and optimizer; returns (step, schedule)."""
    d = torch.load(path, weights_only=False)
    if "scale" in d and not torch.equal(d["scale"], rig.scale):
        raise ValueError("the checkpoint was written with other parameter scales")
    with torch.no_grad():
        rig.params.copy_(d["params"])
    optimizer.load_state_dict(d["optimizer"])
    return d["step"], SeedSchedule(**d["schedule"])
