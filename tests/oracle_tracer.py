"""A stand-in for lighttrace.Tracer backed by the CPU oracle (tests only):
lets the optimisation layer's host logic run without a GPU."""
import numpy as np

import oracle


class OracleTracer:
    def __init__(self):
        self.calls = []

    def upload_scene(self, scene):
        self.sc = scene
        return scene.n_texels

    def set_target(self, E_target, alpha=None):
        self.target = np.asarray(E_target, np.float64)
        self.alpha = np.ones_like(self.target) if alpha is None else np.asarray(alpha, np.float64)

    def set_lights(self, lights):
        self.L = np.array(lights, np.float64)

    def trace_forward(self, seed, n_photons, max_hits, begin=0, end=None):
        self.calls.append(("forward", seed, self.L.copy()))
        self.E = oracle.forward(self.sc, self.L, seed, n_photons, max_hits, begin=begin, end=end, threads=1)["E"]

    def loss(self):
        O, self.w = oracle.loss(self.sc, self.E, self.target, self.alpha)
        return O

    def trace_adjoint(self, seed, n_photons, max_hits, begin=0, end=None, out=None):
        self.calls.append(("adjoint", seed, self.L.copy()))
        g, _ = oracle.adjoint(self.sc, self.L, seed, n_photons, max_hits, self.w, begin=begin, end=end, threads=1)
        return g
