"""What the trained surrogate gains over the method without it: the same
lighting design problem solved by adjoint light tracing alone, and by a
surrogate warm start followed by the tracer. The tracer judges both with a
noise-free estimate of the relative objective."""
import numpy as np
import pytest

from paper_2310_02043_gb300 import _build, scenes, warmstart
from paper_2310_02043_gb300.lighttrace import Tracer

pytestmark = pytest.mark.gpu
HITS = 5


def test_surrogate_warm_start_reaches_the_target_loss_sooner():
    _build.build()
    sc = scenes.office(seed=0, pitch=0.2)
    tr = Tracer(0)
    tr.upload_scene(sc)
    area = tr.texel_areas()
    sg, info = warmstart.fit(tr, n_solves=1024, photons=1 << 19, hits=HITS, steps=600, batch=1 << 16)
    assert np.mean(info["losses"][-20:]) < 0.2 * np.mean(info["losses"][:5])
    start = scenes.office_lights(0)
    truth = scenes.perturb_lights_in_plane(start, 3)
    tr.set_lights(truth)
    tr.trace_forward(77, 1 << 24, HITS)
    target = tr.irradiance()
    thr = 3e-3
    plain_s, plain_hist, _ = warmstart.time_to_loss(
        tr, sc, start, target, [("tracer", 1 << 21, 400, 0.02)], thr, area, eval_photons=1 << 22, max_seconds=20)
    prob = warmstart.SurrogateProblem(sg, target)
    warm_s, warm_hist, _ = warmstart.time_to_loss(
        tr, sc, start, target, [("surrogate", prob, 200, 0.02), ("tracer", 1 << 21, 400, 0.02)], thr, area,
        eval_photons=1 << 22, max_seconds=20)
    info = dict(plain=plain_s, warm=warm_s, plain_last=plain_hist[-1], warm_last=warm_hist[-1],
                start=warmstart.relative_loss(tr, start, target, area, 1 << 22, HITS, 5))
    assert warm_s is not None, info
    assert plain_s is None or warm_s < 0.5 * plain_s, info
    # the surrogate's gradients point downhill in the tracer's objective
    assert warm_hist[0][3] < 0.7 * info["start"], info
    tr.close()
    sg.close()
