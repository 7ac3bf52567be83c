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


class OracleFixedTracer:
    """A stand-in for lighttrace.Tracer that keeps its sums the way the
    library does, for host-side tests of multi-rank code: the forward pass
    adds every deposit as round(Phi S) to an int64 texel array (exact, so
    photon partitions add up bit for bit), the objective reads the (possibly
    all-reduced) integers, and the adjoint keeps exact per-light sums of
    every photon's term rounded to 2^-64 / G, with G = 2^-e from the largest
    weight. Deposits and terms come from the oracle's path records."""

    def __init__(self, scale_exp: int = 40):
        self.S = float(2 ** scale_exp)

    def upload_scene(self, scene):
        self.sc = scene
        self.A = oracle.texel_areas(scene)
        self.q = np.zeros(scene.n_texels, np.int64)
        return scene.n_texels

    def set_target(self, E_target, alpha=None):
        self.target = np.asarray(E_target, np.float64)

    def set_lights(self, lights):
        self.L = np.array(lights, np.float64)

    def trace_forward(self, seed, n_photons, max_hits, begin=0, end=None):
        end = n_photons if end is None else end
        tri, tex, phi = oracle.paths(self.sc, self.L, seed, n_photons, max_hits, begin, end - begin, threads=1,
                                     flux=True)
        self.q[:] = 0
        ok = tex >= 0
        np.add.at(self.q, tex[ok], np.rint(phi[ok] * self.S).astype(np.int64))

    def loss(self, out=None):
        E = self.q.astype(np.float64) / self.S / self.A
        O, self.w = oracle.loss(self.sc, E, self.target, np.ones(self.sc.n_texels))
        return O

    def trace_adjoint(self, seed, n_photons, max_hits, begin=0, end=None, out=None):
        from fractions import Fraction

        from paper_2310_02043_gb300.lighttrace import gradient_from_fixed
        end = n_photons if end is None else end
        _, _, c = oracle.paths(self.sc, self.L, seed, n_photons, max_hits, begin, end - begin, threads=1, w=self.w)
        wmax = float(np.max(np.abs(self.w)))
        self.G = 2.0 ** -np.floor(np.log2(wmax)) if wmax > 0 else 1.0
        sizes = np.full(self.L.shape[0], n_photons // self.L.shape[0]) + (np.arange(self.L.shape[0])
                                                                          < n_photons % self.L.shape[0])
        lights = np.searchsorted(np.cumsum(sizes), np.arange(begin, end), side="right")
        unit = Fraction(2 ** 64) * Fraction(self.G)
        self.fixed = np.empty((self.L.shape[0], 8), dtype=object)
        self.fixed[...] = 0
        for p in range(c.shape[0]):
            for k in range(8):
                if c[p, k] != 0.0:
                    self.fixed[lights[p], k] += round(Fraction(c[p, k]) * unit)
        g = gradient_from_fixed(self.fixed, self.G)
        if out is not None:
            out[...] = g
            return out
        return g

    def gradient_fixed(self):
        sums = np.empty(self.fixed.shape + (2,), np.int64)
        for idx in np.ndindex(self.fixed.shape):
            v = int(self.fixed[idx])
            lo = v & ((1 << 64) - 1)
            sums[idx] = (lo - (1 << 64) if lo >= (1 << 63) else lo, v >> 64)
        return sums, self.G
