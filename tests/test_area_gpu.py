"""Rectangular area lights on the GPU against the oracle: irradiance, photon
paths and gradients (supplement Eq. S.15-S.16), mixed with spots and point
lights; and the argument checks of the light record."""
import numpy as np
import pytest

import oracle
from paper_2310_02043_gb300 import _build, scenes
from paper_2310_02043_gb300.lighttrace import LtError, Tracer
from tests.test_gpu_parity import _adjoint_case, _check_irradiance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tr():
    _build.build()
    t = Tracer(0)
    yield t
    t.close()


def _cornell_area_lights():
    return scenes.make_lights([
        scenes.area_light((0.5, 0.5, 0.98), 0.3, -np.pi / 2 + 0.05, 1.5, 0.25, 0.15),
        scenes.area_light((0.25, 0.7, 0.6), 1.1, -0.3, 0.8, 0.1, 0.2),
        scenes.spot_light((0.7, 0.3, 0.95), 0.5, -1.3, 1.0, 0.3, 0.6),
        scenes.point_light((0.3, 0.3, 0.5), 0.4)])


def test_area_forward_matches_oracle(tr):
    sc, L = scenes.cornell_box(res=8), _cornell_area_lights()      # ~2800 deposits per texel
    n, hits, seed = 1 << 20, 3, 5
    tr.upload_scene(sc)
    tr.set_lights(L)
    tr.trace_forward(seed, n, hits)
    E = tr.irradiance().astype(np.float64)
    ref = oracle.forward(sc, L, seed, n, hits, counts=True)
    assert _check_irradiance(sc, E, ref) > 100
    assert abs(tr.stats()["segments_forward"] - ref["segments"]) <= 1e-4 * ref["segments"]


def test_area_paths_match_oracle(tr):
    sc, L = scenes.cornell_box(res=32), _cornell_area_lights()
    n, hits, seed = 1 << 18, 3, 6
    tr.upload_scene(sc)
    tr.set_lights(L)
    tri, tex = tr.debug_paths(seed, n, hits, 0, n)
    tri_o, tex_o = oracle.paths(sc, L, seed, n, hits, 0, n)
    same = np.all(tri == tri_o, axis=1) & np.all(tex == tex_o, axis=1)
    assert same.mean() >= 0.999, same.mean()


def test_area_adjoint_matches_oracle(tr):
    sc, L = scenes.cornell_box(res=32), _cornell_area_lights()
    Lt = L.copy()
    Lt[:, 1:3] += np.random.default_rng(4).normal(0, 0.03, (L.shape[0], 2))
    target = oracle.forward(sc, Lt, 77, 1 << 16, 3)["E"].astype(np.float32)
    # uniform-hemisphere emission makes grazing first hits common, where the
    # 1/cos_1 of Eq. 14 amplifies float rounding in single photons' terms
    g = _adjoint_case(tr, sc, L, target, 1 << 18, 3, 8, term_tol=5e-2)
    assert np.all(g[:2, 6:] == 0)                  # area lights: no cone slots
    assert np.all(np.abs(g[:2, :6]) > 0)


def test_area_light_arguments(tr):
    sc = scenes.cornell_box(res=8)
    tr.upload_scene(sc)
    bad = scenes.make_lights([scenes.area_light((0.5, 0.5, 0.9), 0.0, -1.5, 1.0, 0.0, 0.2)])
    with pytest.raises(LtError):
        tr.set_lights(bad)
    bad[0, 7], bad[0, 8] = 0.2, float("inf")
    with pytest.raises(LtError):
        tr.set_lights(bad)
