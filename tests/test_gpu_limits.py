"""Edge sizes on the GPU against the oracle: the maximum light count
(LT_MAX_LIGHTS luminaires of all three kinds, a photon budget that does not
divide evenly), the maximum path length (64 hits in a closed box, against
the closed-form energy), the arguments beyond the limits, a failed scene
upload (host allocation failure, injected on the host), and the tracing
kernels' give-up limit run out on purpose (the kernels end the rays and
report; nothing waits or traps)."""
import numpy as np
import pytest

import oracle
from paper_2310_02043_gb300 import _build, scenes
from paper_2310_02043_gb300.lighttrace import LtError, Tracer
from tests import parity
from tests.test_gpu_parity import _check_irradiance

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
    # about 1000 photons per light and random weights of either sign: one
    # grazing first hit (1/cos_1 amplifies float rounding in that photon's
    # term) or one photon whose path parted can move a light's sum by
    # ~1e-3..1e-2 of the largest component (raw: measured 2.2e-2), so the
    # bounds here are 1e-2 per light with the parted photons exchanged and
    # 5e-2 raw; every photon's term is checked on its own inside
    # parity.check_gradient
    m = (1 << 20) + 5
    g = tr.trace_adjoint(seed, m, hits)
    g_ref, _ = oracle.adjoint(sc, L, seed, m, hits, w.astype(np.float64))
    parity.check_gradient(tr, sc, L, seed, m, hits, w.astype(np.float64), g, g_ref, raw_rtol=5e-2, rtol=1e-2,
                          term_tol=5e-2)
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
    # a pass covers at most 2^32 - 1 photons (the kernels count a pass's
    # photons in 32 bits); larger ranges are refused before any launch, and a
    # small range far into a larger budget is fine
    with pytest.raises(LtError, match="2\\^32"):
        tr.trace_forward(1, 1 << 33, 3, 0, 1 << 32)
    with pytest.raises(LtError, match="2\\^32"):
        tr.batch_setup([2, 1], 1 << 31, 3)
    tr.trace_forward(1, 1 << 33, 3, (1 << 33) - 4096, 1 << 33)
    assert tr.stats()["segments_forward"] > 0


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


def test_step_limit_runs_out_and_the_context_recovers(tr):
    """With a give-up limit of one node visit per ray every ray of the office
    (a 5-level BVH) gives up: the kernels end those rays, the next
    synchronising call reports LT_ERR_TIMEOUT once, and after the default is
    restored the same passes give the same results as before."""
    from paper_2310_02043_gb300.lighttrace import LT_ERR_TIMEOUT
    sc, L = scenes.office(seed=0, pitch=0.1), scenes.office_lights(0)
    n, hits = 1 << 16, 5
    tr.upload_scene(sc)
    tr.set_lights(L)
    tr.trace_forward(5, n, hits)
    q_ref = tr.texel_sums().copy()
    w = scenes.random_weights(sc.n_texels, seed=3)
    tr.set_adjoint_weights(w)
    g_ref = tr.trace_adjoint(6, n, hits)
    with pytest.raises(LtError):
        tr.set_step_limit(-1)
    tr.set_step_limit(1)
    tr.trace_forward(5, n, hits)
    with pytest.raises(LtError) as e:
        tr.stats()
    assert e.value.status == LT_ERR_TIMEOUT
    tr.stats()                                       # reported once, then cleared
    tr.set_adjoint_weights(w)
    with pytest.raises(LtError) as e:
        tr.trace_adjoint(6, n, hits)
    assert e.value.status == LT_ERR_TIMEOUT
    tr.set_step_limit(0)
    tr.trace_forward(5, n, hits)
    assert tr.stats()["segments_forward"] == n * hits
    assert np.array_equal(tr.texel_sums(), q_ref)
    tr.set_adjoint_weights(w)
    assert np.array_equal(tr.trace_adjoint(6, n, hits), g_ref)
