"""Batched designs: one launch traces several candidate designs with uneven
light counts. Each design must match the oracle with that design's Philox
word (texels, objective, gradient), and equal a single-design pass with the
same word; graph replay must equal eager issue."""
import numpy as np
import pytest

import oracle
from paper_2310_02043_gb300 import _build, autotune, scenes
from paper_2310_02043_gb300.lighttrace import Tracer
from tests import parity

pytestmark = pytest.mark.gpu

N, HITS = 1 << 16, 5
COUNTS = [4, 7, 1, 12, 3]


def _designs():
    rng = np.random.default_rng(8)
    base = scenes.office_lights(0)
    designs = []
    for d, n in enumerate(COUNTS):
        pick = rng.choice(len(base), size=n, replace=False)
        designs.append(scenes.perturb_lights(base[pick], seed=100 + d, pos_sigma=0.3, angle_sigma=0.1))
    return designs


@pytest.fixture(scope="module")
def setup():
    _build.build()
    sc = scenes.office(seed=0, pitch=0.1)
    target = oracle.forward(sc, scenes.office_lights(0), 50, 1 << 15, HITS)["E"].astype(np.float32)
    tr = Tracer(0)
    tr.upload_scene(sc)
    tr.set_target(target)
    yield tr, sc, target, _designs()
    tr.close()


def _single(tr, lights, design, seed_f, seed_a):
    tr.set_design(design)
    tr.set_lights(lights)
    tr.trace_forward(seed_f, N, HITS)
    O = tr.loss()
    E = tr.irradiance()
    g = tr.trace_adjoint(seed_a, N, HITS)
    return E, O, g


def test_batch_designs_equal_single_design_passes(setup):
    # A batch sizes one fixed-point scale (a power of two) for its brightest
    # design, a single pass for its own lights: the same paths, the same
    # irradiance up to rounding of that scale.
    tr, sc, target, designs = setup
    tr.batch_setup(COUNTS, N, HITS)
    tr.batch_set_lights(np.concatenate(designs))
    loss, grad = tr.batch_step(11, 12)
    off = 0
    for d, L in enumerate(designs):
        Eb = tr.batch_irradiance(d).astype(np.float64)
        E, O, g = _single(tr, L, d, 11, 12)
        E = E.astype(np.float64)
        diff = np.abs(Eb - E)
        info = dict(design=d, n_diff=int((diff > 0).sum()), max_rel=float((diff / np.maximum(E, 1e-30)).max()),
                    sum_b=float(Eb.sum()), sum_s=float(E.sum()))
        # each deposit rounds to a quantum of 1/S; a texel with a few faint
        # deposits differs by a few quanta, far below 1e-9 of the brightest
        assert np.all(diff <= 1e-6 * np.abs(E) + 1e-9 * E.max()), info
        assert np.mean(diff == 0) > 0.999, info
        assert loss[d] == pytest.approx(O, rel=1e-9), d
        gb = grad[off:off + len(L)]
        # the batch's fixed-point texel scale differs from the single pass's,
        # so do the weights by its rounding, and so the gradients
        assert np.allclose(gb, g, rtol=1e-5, atol=1e-6 * np.abs(g).max()), d
        off += len(L)
    tr.set_design(0)


def test_batch_with_point_spot_and_area_lights(setup):
    # designs of mixed luminaire kinds (area lights draw their origin from
    # Philox lanes 2-3): each design equals its single-design pass
    tr, sc, target, designs = setup
    mixed = [scenes.make_lights([scenes.point_light((4.0, 3.0, 2.7), 30.0),
                                 scenes.area_light((10.0, 5.0, 2.95), 0.0, -np.pi / 2, 400.0, 1.2, 0.6)]),
             scenes.make_lights([scenes.area_light((6.0, 7.0, 2.95), 0.5, -np.pi / 2 + 0.1, 300.0, 0.6, 0.6),
                                 scenes.spot_light((15.0, 4.0, 2.8), 0.3, -1.4, 40.0, 0.6, 1.0),
                                 scenes.area_light((3.0, 2.0, 2.95), 1.0, -np.pi / 2, 200.0, 1.0, 0.3)])]
    counts = [len(L) for L in mixed]
    tr.batch_setup(counts, N, HITS)
    tr.batch_set_lights(np.concatenate(mixed))
    loss, grad = tr.batch_step(31, 32)
    off = 0
    for d, L in enumerate(mixed):
        Eb = tr.batch_irradiance(d).astype(np.float64)
        E, O, g = _single(tr, L, d, 31, 32)
        E = E.astype(np.float64)
        diff = np.abs(Eb - E)
        assert np.all(diff <= 1e-6 * np.abs(E) + 1e-9 * E.max()), d
        assert loss[d] == pytest.approx(O, rel=1e-9), d
        gb = grad[off:off + len(L)]
        assert np.allclose(gb, g, rtol=1e-5, atol=1e-6 * np.abs(g).max()), d
        # slots that exist for each kind: orientation for spots and area
        # lights, cone angles for spots only
        kinds = L[:, 0]
        assert np.all(np.abs(gb[:, [0, 1, 2, 5]]) > 0), d
        assert np.all(np.abs(gb[kinds != scenes.POINT][:, [3, 4]]) > 0), d
        assert np.all(gb[kinds == scenes.POINT][:, [3, 4]] == 0), d
        assert np.all(gb[kinds != scenes.SPOT][:, 6:] == 0), d
        off += len(L)
    tr.set_design(0)


def test_batch_matches_the_oracle(setup):
    # Three designs of uneven light counts (1, 3 and 5) mixing area, point
    # and spot lights, 2^18 photons each, in one batch step. Per design
    # against the oracle with the design's Philox word: every texel (the
    # photons whose paths parted accounted for on both sides), the objective
    # to 1e-4, and the gradient to 1e-3 from the adjoint weights the batch
    # itself formed (rebuilt here from its integer texel sums as its loss
    # kernel forms them).
    tr, sc, target, _ = setup
    base = scenes.office_lights(0)
    designs = [scenes.make_lights([scenes.area_light((10.0, 5.0, 2.95), 0.0, -np.pi / 2, 400.0, 1.2, 0.6)]),
               scenes.make_lights([scenes.point_light((4.0, 3.0, 2.7), 30.0),
                                   scenes.spot_light((15.0, 4.0, 2.8), 0.3, -1.4, 40.0, 0.6, 1.0),
                                   scenes.area_light((3.0, 2.0, 2.95), 1.0, -np.pi / 2, 200.0, 1.0, 0.3)]),
               scenes.perturb_lights(base[[0, 3, 5, 9, 14]], seed=7, pos_sigma=0.3, angle_sigma=0.1)]
    n, sf, sa = 1 << 18, 41, 42
    tr.batch_setup([len(L) for L in designs], n, HITS)
    tr.batch_set_lights(np.concatenate(designs))
    loss, grad = tr.batch_step(sf, sa)
    S = tr.stats()["fixed_point_scale"]
    A32 = tr.texel_areas().astype(np.float64)
    off = 0
    try:
        for d, L in enumerate(designs):
            q = tr.batch_texel_sums(d)
            tr.set_design(d)
            tr.set_lights(L)
            info = parity.check_every_texel(tr, sc, L, sf, n, HITS, 0, n, q, S, design=d)
            assert info["texels"] == sc.n_texels and info["lit"] > 0.5 * sc.n_texels, (d, info)
            ref = oracle.forward(sc, L, sf, n, HITS, design=d)
            O_ref, _ = oracle.loss(sc, ref["E"], target, np.ones(sc.n_texels))
            assert abs(loss[d] - O_ref) <= 1e-4 * O_ref, (d, loss[d], O_ref)
            w = (q.astype(np.float64) * (1.0 / S) / A32 - target.astype(np.float64)).astype(np.float32)
            tr.set_adjoint_weights(w)
            g_ref, _ = oracle.adjoint(sc, L, sa, n, HITS, w.astype(np.float64), design=d)
            parity.check_gradient(tr, sc, L, sa, n, HITS, w.astype(np.float64), grad[off:off + len(L)], g_ref,
                                  design=d)
            off += len(L)
    finally:
        tr.set_design(0)


def test_graph_replay_equals_eager(setup):
    tr, sc, target, designs = setup
    tr.batch_setup(COUNTS, N, HITS)
    assert tr.batch_stream() != 0
    lights = np.concatenate(designs)
    for step, shift in enumerate([0.0, 0.05, -0.03]):
        L = lights.copy()
        L[:, 1] += shift
        tr.batch_set_lights(L)
        lg, gg = tr.batch_step(20 + step, 40 + step, use_graph=True)
        sg = tr.stats()
        le, ge = tr.batch_step(20 + step, 40 + step, use_graph=False)
        se = tr.stats()
        assert np.array_equal(lg, le) and np.array_equal(gg, ge), step
        # the step's own segment counts, all designs, both passes
        assert sg["segments_forward"] == se["segments_forward"] > sum(COUNTS) and sg["segments_adjoint"] > 0
        assert sg["photons_forward"] == N * len(COUNTS)


def test_design_word_matches_the_oracle(setup):
    tr, sc, target, designs = setup
    L = designs[3]
    tr.set_design(3)
    tr.set_lights(L)
    tr.trace_forward(9, N, HITS)
    E = tr.irradiance().astype(np.float64)
    tr.set_design(0)
    ref = oracle.forward(sc, L, 9, N, HITS, design=3)
    other = oracle.forward(sc, L, 9, N, HITS, design=0)
    A = oracle.texel_areas(sc)
    tot, tot_ref = np.sum(A * E), np.sum(A * ref["E"])
    assert abs(tot - tot_ref) <= 1e-4 * tot_ref
    # the word changes the random numbers: design 0 gives other texels
    assert np.abs(E - ref["E"]).sum() < 0.1 * np.abs(E - other["E"]).sum()


def test_autotuned_shape_keeps_the_results(setup, tmp_path):
    tr, sc, target, designs = setup
    tr.batch_setup(COUNTS, N, HITS)
    tr.batch_set_lights(np.concatenate(designs))
    tr.set_launch(256, 0, 200 * 1024)
    ref_loss, ref_grad = tr.batch_step(3, 4)
    q0 = tr.batch_texel_sums(2)
    best, res = autotune.tune(tr, lambda: tr.batch_step(3, 4, use_graph=True), "office-test",
                              cache_path=str(tmp_path / "t.json"), repeats=2)
    assert best in res and len(res) >= 4
    loss, grad = tr.batch_step(3, 4, use_graph=True)
    assert np.array_equal(tr.batch_texel_sums(2), q0)
    assert np.allclose(loss, ref_loss, rtol=1e-12)
    # exact gradient sums: the launch shape does not change a bit
    assert np.array_equal(grad, ref_grad)
    tr.set_launch(256, 0, 200 * 1024)
