"""The GPU path on the scenes where the oracle is pinned to closed forms,
so that the chain from kernel to mathematics is short:

* inside a diffuse sphere over 8 hits (every orientation of the mesh, the
  1/(1 - rho) interreflection): irradiance against the oracle on the same
  paths, and the deposited energy against the geometric series over the hits
  each GPU photon made;
* a point light over a plane under a square occluder: the GPU adjoint
  (Alg. 2, Eq. 11 and 14, first hit held fixed) against central differences
  of the quadrature objective with visibility frozen, on every axis, directly
  and without the oracle."""
import numpy as np
import pytest

import oracle
from paper_2310_02043_gb300 import _build, scenes
from paper_2310_02043_gb300.lighttrace import Tracer
from tests.test_gpu_parity import _check_irradiance
from tests.test_oracle_shadow import HALF, OC, OH, RES, ZO, _floor_irradiance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tr():
    _build.build()
    t = Tracer(0)
    yield t
    t.close()


def test_sphere_interreflection(tr):
    rho, B, n, seed = 0.5, 8, 1 << 19, 11
    sc = scenes.icosphere(radius=1.0, subdiv=3, albedo=rho)
    L = scenes.make_lights([scenes.point_light((-0.25, 0.4, 0.1), 1.0)])
    tr.upload_scene(sc)
    tr.set_lights(L)
    tr.trace_forward(seed, n, B)
    E = tr.irradiance().astype(np.float64)
    ref = oracle.forward(sc, L, seed, n, B, counts=True)
    assert _check_irradiance(sc, E, ref) == sc.n_texels
    tri, _ = tr.debug_paths(seed, n, B, 0, n)
    hits = np.sum(tri >= 0, axis=1)
    assert np.all(hits >= 1) and np.sum(B - hits) <= 1e-5 * n * B
    assert tr.stats()["segments_forward"] == np.sum(np.minimum(hits + 1, B))
    geo = np.cumsum(rho ** np.arange(B))                  # 1 + rho + ... + rho^(h-1)
    A = oracle.texel_areas(sc)
    assert np.sum(A * E) == pytest.approx(4 * np.pi / n * np.sum(geo[hits - 1]), rel=1e-6)


def test_adjoint_is_the_frozen_visibility_derivative(tr):
    sc = scenes.occluded_plane(HALF, RES, ZO, OC, OH)
    L = scenes.make_lights([scenes.point_light((0.2, 0.1, 1.0), 1.0)])
    x0 = L[0, 1:4].copy()
    A = oracle.texel_areas(sc)
    nf = RES * RES
    w = np.zeros(sc.n_texels, np.float32)
    w[:nf] = _floor_irradiance(x0, x0)

    def objective(x):
        E = _floor_irradiance(x, x0)                          # visibility frozen at x0
        return 0.5 * np.sum(A[:nf] * E * E)

    tr.upload_scene(sc)
    tr.set_lights(L)
    tr.set_adjoint_weights(w)
    n, batches, seed = 1 << 24, 16, 3
    per = n // batches
    parts = np.array([tr.trace_adjoint(seed, n, 1, k * per, (k + 1) * per)[0] * batches for k in range(batches)])
    G, sigma = parts.mean(0), parts.std(0, ddof=1) / np.sqrt(batches)
    for axis in range(3):
        xp, xm = x0.copy(), x0.copy()
        xp[axis] += 1e-2
        xm[axis] -= 1e-2
        fd = (objective(xp) - objective(xm)) / 2e-2
        assert abs(G[axis] - fd) <= 4.0 * sigma[axis] + 2e-3 * abs(fd), (axis, G[axis], fd, sigma[axis])
