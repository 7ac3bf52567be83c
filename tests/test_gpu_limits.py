"""Edge sizes on the GPU against the oracle: the maximum light count
(LT_MAX_LIGHTS luminaires of all three kinds, a photon budget that does not
divide evenly), the maximum path length (64 hits in a closed box, against
the closed-form energy), the arguments beyond the limits, and a failed scene
upload (host allocation failure, injected on the host)."""
import numpy as np
import pytest

import oracle
from paper_2310_02043_gb300 import _build, scenes
from paper_2310_02043_gb300.lighttrace import LtError, Tracer
from tests.test_gpu_parity import _check_grad, _check_irradiance

pytestmark = pytest.mark.gpu
MAX_LIGHTS = 1024


@pytest.fixture(scope="module")
def tr():
    _build.build()
    t = Tracer(0)
    yield t
    t.close()


def test_maximum_light_count(tr):
    sc = scenes.cornell_box(res=8)
    L = scenes.random_lights(MAX_LIGHTS, seed=4)
    n, hits, seed = 1_000_003, 3, 12                 # 976 or 977 photons per light
    tr.upload_scene(sc)
    tr.set_lights(L)
    tr.trace_forward(seed, n, hits)
    E = tr.irradiance().astype(np.float64)
    ref = oracle.forward(sc, L, seed, n, hits, counts=True)
    assert _check_irradiance(sc, E, ref) > 100
    w = scenes.random_weights(sc.n_texels, seed=6)
    tr.set_adjoint_weights(w)
    # about 1000 photons per light: one grazing first hit (1/cos_1 amplifies
    # float rounding in that photon's term) can still move a light's sum by
    # ~1e-3..1e-2, so the per-light bound here is 1e-2; every photon's term is
    # checked on its own inside _check_grad
    m = (1 << 20) + 5
    g = tr.trace_adjoint(seed, m, hits)
    g_ref, _ = oracle.adjoint(sc, L, seed, m, hits, w.astype(np.float64))
    _check_grad(tr, sc, L, seed, m, hits, w.astype(np.float64), g, g_ref, rtol=1e-2, term_tol=5e-2)
    assert g.shape == (MAX_LIGHTS, 8)


def test_maximum_path_length(tr):
    rho, I, hits = 0.9, 1.0, 64
    sc = scenes.closed_cube(res=4, albedo=rho)
    L = scenes.make_lights([scenes.point_light((0.4, 0.55, 0.6), I)])
    n = 1 << 16
    tr.upload_scene(sc)
    tr.set_lights(L)
    tr.trace_forward(3, n, hits)
    segs = tr.stats()["segments_forward"]
    assert n * hits - segs <= 1e-5 * n * hits           # a closed box keeps (almost) every path
    A = tr.texel_areas().astype(np.float64)
    total = float(np.sum(A * tr.irradiance()))
    r32 = float(np.float32(rho))
    expected = 4 * np.pi * I * (1 - r32 ** hits) / (1 - r32)
    assert abs(total - expected) <= 1e-4 * expected + (n * hits - segs) / n * 4 * np.pi * I
    ref = oracle.forward(sc, L, 3, n, hits, counts=True)
    _check_irradiance(sc, tr.irradiance().astype(np.float64), ref)


def test_limits_are_rejected(tr):
    sc = scenes.cornell_box(res=4)
    tr.upload_scene(sc)
    with pytest.raises(LtError):
        tr.set_lights(scenes.random_lights(MAX_LIGHTS + 1, seed=1))
    tr.set_lights(scenes.random_lights(3, seed=1))
    for bad in (0, 65):
        with pytest.raises(LtError):
            tr.trace_forward(1, 1000, bad)


def test_power_beyond_the_fixed_point_range(tr):
    from paper_2310_02043_gb300.lighttrace import LT_ERR_OVERFLOW
    sc = scenes.cornell_box(res=4)
    tr.upload_scene(sc)
    L = scenes.make_lights([scenes.point_light((0.5, 0.5, 0.5), 1e60)])
    tr.set_lights(L)
    with pytest.raises(LtError) as e:
        tr.trace_forward(1, 1000, 3)
    assert e.value.status == LT_ERR_OVERFLOW
    tr.set_lights(scenes.make_lights([scenes.point_light((0.5, 0.5, 0.5), 1e30)]))
    tr.trace_forward(1, 1000, 3)                          # large but representable
    assert np.isfinite(tr.irradiance()).all()



def test_failed_scene_upload_keeps_the_previous_scene(tr, monkeypatch):
    """A host allocation failure inside lt_upload_scene (injected) is
    LT_ERR_OOM with a message; the context keeps the scene it had, traces it
    bit for bit as before, and takes the next upload."""
    from paper_2310_02043_gb300.lighttrace import LT_ERR_OOM
    sc = scenes.cornell_box(res=8)
    L = scenes.make_lights([scenes.point_light((0.5, 0.5, 0.9), 1.0)])
    tr.upload_scene(sc)
    tr.set_lights(L)
    tr.trace_forward(5, 1 << 16, 3)
    q = tr.texel_sums().copy()
    monkeypatch.setenv("LT_FAULT_HOST_ALLOC", "1")
    with pytest.raises(LtError) as e:
        tr.upload_scene(scenes.cornell_box(res=16))
    assert e.value.status == LT_ERR_OOM and "host memory" in str(e.value)
    monkeypatch.delenv("LT_FAULT_HOST_ALLOC")
    tr.trace_forward(5, 1 << 16, 3)
    assert np.array_equal(tr.texel_sums(), q)
    big = scenes.cornell_box(res=16)
    assert tr.upload_scene(big) == big.n_texels
