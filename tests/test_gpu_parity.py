"""GPU path vs the CPU oracle on the same seeded inputs (calls go through the C ABI).

Tolerances (the path computes in FP32, the oracle in FP64; both take the
hit/texel decisions in float, so a small fraction of paths can still part
ways near triangle or texel edges):
  * irradiance: sum_t A_t E_t to 1e-4 relative; E_t to 1e-3 relative on every
    texel that received at least 1e3 deposits; and every texel to 1e-5 once
    the photons whose paths parted are removed from both sides
    (``parity.check_every_texel``);
  * objective O to 1e-4 relative;
  * gradients: every component to 1e-3 relative, against
    max(|g_oracle|, 1e-3 max|g_oracle|), as the GPU returns it and again with
    the parted photons' terms exchanged (``parity.check_gradient``);
  * fixed-point texel sums are bit-identical across launch shapes and reruns.
"""
import numpy as np
import pytest

import oracle
from paper_2310_02043_gb300 import _build, scenes
from paper_2310_02043_gb300.lighttrace import LtError, Tracer, gradient_from_fixed
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tr():
    _build.build()
    t = Tracer(0)
    yield t
    t.close()


def _forward(tr, sc, lights, seed, n, hits, begin=0, end=None):
    tr.upload_scene(sc)
    tr.set_lights(lights)
    tr.trace_forward(seed, n, hits, begin, n if end is None else end)
    return tr.irradiance().astype(np.float64), tr.stats()


def _check_irradiance(sc, E, ref, min_count=1000):
    """Aggregate to 1e-4; 1e-3 per texel on texels with >= min_count oracle
    deposits. Returns how many texels the per-texel gate covered."""
    A = oracle.texel_areas(sc)
    tot, tot_ref = np.sum(A * E), np.sum(A * ref["E"])
    assert abs(tot - tot_ref) <= 1e-4 * tot_ref, (tot, tot_ref)
    m = ref["count"] >= min_count
    rel = np.abs(E[m] - ref["E"][m]) / ref["E"][m]
    bad = np.nonzero(rel > 1e-3)[0]
    assert len(bad) == 0, f"{len(bad)} of {m.sum()} texels beyond 1e-3 (worst {rel.max():.3g})"
    return int(m.sum())


def _every_texel(tr, sc, L, seed, n, hits, begin=0, end=None):
    end = n if end is None else end
    st = tr.stats()
    info = parity.check_every_texel(tr, sc, L, seed, n, hits, begin, end, tr.texel_sums(), st["fixed_point_scale"])
    assert info["texels"] == sc.n_texels
    return info


def test_cornell_forward_matches_oracle(tr):
    sc, L = scenes.cornell_box(res=32), scenes.cornell_lights()
    n, hits, seed = 1 << 20, 3, 2
    E, st = _forward(tr, sc, L, seed, n, hits)
    ref = oracle.forward(sc, L, seed, n, hits, counts=True)
    assert _check_irradiance(sc, E, ref) > 100
    assert abs(st["segments_forward"] - ref["segments"]) <= 1e-4 * ref["segments"]
    info = _every_texel(tr, sc, L, seed, n, hits)
    assert info["lit"] > 0.95 * sc.n_texels, info["lit"]


def test_cornell_paths_match_oracle(tr):
    sc, L = scenes.cornell_box(res=32), scenes.cornell_lights()
    n, hits, seed = 1 << 20, 3, 2
    tr.upload_scene(sc)
    tr.set_lights(L)
    tri, tex = tr.debug_paths(seed, n, hits, 1000, 20000)
    tri_o, tex_o = oracle.paths(sc, L, seed, n, hits, 1000, 20000)
    same = np.all(tri == tri_o, axis=1) & np.all(tex == tex_o, axis=1)
    assert same.mean() >= 0.999, same.mean()


def test_office_forward_matches_oracle(tr):
    sc, L = scenes.office(seed=0, pitch=0.1), scenes.office_lights(0)
    n, hits, seed = 1 << 17, 5, 3
    E, st = _forward(tr, sc, L, seed, n, hits)
    ref = oracle.forward(sc, L, seed, n, hits, counts=True)
    _check_irradiance(sc, E, ref, min_count=1000)
    # closed room: every photon makes exactly `hits` segments
    assert st["segments_forward"] == n * hits == ref["segments"]
    info = _every_texel(tr, sc, L, seed, n, hits)
    assert info["lit"] > 0.8 * sc.n_texels, info["lit"]


def test_office_benchmark_texels_match_oracle(tr):
    # The benchmark's scene as it is benchmarked: 2 cm texels (3.2 M), 16
    # spots, 5 hits; every texel compared, the parted photons accounted for.
    sc, L = scenes.office(seed=0, pitch=0.02), scenes.office_lights(0)
    n, hits, seed = 1 << 24, 5, 2
    begin, end = 5_000_000, 5_000_000 + (1 << 20)
    tr.upload_scene(sc)
    tr.set_lights(L)
    tr.trace_forward(seed, n, hits, begin, end)
    assert tr.stats()["segments_forward"] == (end - begin) * hits
    info = _every_texel(tr, sc, L, seed, n, hits, begin, end)
    assert info["lit"] > 0.4 * sc.n_texels, info["lit"]


def test_office_coarse_texels_with_many_deposits(tr):
    # The per-texel gate as stated (1e-3 on texels with >= 1e3 deposits) with
    # enough deposits per texel for it to cover most of the scene: 50 cm
    # texels (6450), 2^21 photons x 5 hits. A photon whose float path parted
    # from the double one moves its texels by its whole deposit, which for a
    # direct spot photon among interreflected ones can exceed 1e-3 of a
    # texel's sum; so the raw gate covers the texels no parted photon
    # touched, and every texel is compared exactly once the parted photons
    # are accounted for.
    sc, L = scenes.office(seed=0, pitch=0.5), scenes.office_lights(0)
    n, hits, seed = 1 << 21, 5, 6
    E, st = _forward(tr, sc, L, seed, n, hits)
    info = _every_texel(tr, sc, L, seed, n, hits)
    ref = oracle.forward(sc, L, seed, n, hits, counts=True)
    A = oracle.texel_areas(sc)
    assert abs(np.sum(A * E) - np.sum(A * ref["E"])) <= 1e-4 * np.sum(A * ref["E"])
    m = (ref["count"] >= 1000) & ~info["touched"]
    rel = np.abs(E[m] - ref["E"][m]) / ref["E"][m]
    assert np.all(rel <= 1e-3), rel.max()
    assert m.sum() > 0.25 * sc.n_texels, (int(m.sum()), int((ref["count"] >= 1000).sum()))


def test_ragged_range_and_mixed_lights(tr):
    sc = scenes.cornell_box(res=16)
    L = scenes.make_lights([scenes.point_light((0.5, 0.5, 0.9), 1.0),
                            scenes.spot_light((0.3, 0.3, 0.95), 0.3, -1.4, 2.0, 0.0, 0.7),
                            scenes.spot_light((0.7, 0.6, 0.9), 2.0, -1.2, 1.5, 0.3, 0.5)])
    n, hits, seed, b, e = 100_003, 2, 7, 37, 90_001
    E, st = _forward(tr, sc, L, seed, n, hits, b, e)
    ref = oracle.forward(sc, L, seed, n, hits, begin=b, end=e, counts=True)
    _check_irradiance(sc, E, ref, min_count=1000)
    assert st["photons_forward"] == e - b
    info = _every_texel(tr, sc, L, seed, n, hits, b, e)
    assert info["lit"] > 0.9 * sc.n_texels, info


def test_empty_range_and_dark_light(tr):
    sc = scenes.cornell_box(res=8)
    L = scenes.make_lights([scenes.point_light((0.5, 0.5, 0.9), 1.0), scenes.point_light((0.2, 0.2, 0.5), 0.0)])
    E, st = _forward(tr, sc, L, 1, 5000, 3, 2000, 2000)
    assert np.all(E == 0) and st["segments_forward"] == 0
    # the dark light (p_int = 0) deposits nothing; the other light is unchanged
    E, st = _forward(tr, sc, L, 1, 5000, 3)
    ref = oracle.forward(sc, L, 1, 5000, 3, counts=True)
    A = oracle.texel_areas(sc)
    assert abs(np.sum(A * E) - np.sum(A * ref["E"])) <= 1e-4 * np.sum(A * ref["E"])


def test_all_photons_escape(tr):
    sc = scenes.plane(half=1.0, res=4)
    L = scenes.make_lights([scenes.spot_light((0.0, 0.0, 1.0), 0.0, 1.2, 1.0, 0.2, 0.4)])  # points up
    E, st = _forward(tr, sc, L, 1, 4096, 3)
    assert np.all(E == 0) and st["segments_forward"] == 4096


def test_single_triangle_scene_staged_and_through_l1(tr):
    # The smallest scene: one triangle, so the BVH is one node whose only
    # child is a leaf. Both node paths (staged and through L1) trace it; the
    # texel and the gradient match the oracle, and the two paths give the
    # same integer sums.
    b = scenes._Builder()
    b.triangle([-1.0, -1.0, 0.0], [1.5, -1.0, 0.0], [-1.0, 1.5, 0.0], 0.6)
    sc = b.build("one triangle")
    L = scenes.make_lights([scenes.point_light((0.0, 0.0, 0.7), 1.0)])
    n, hits, seed = 1 << 16, 3, 6
    E, st = _forward(tr, sc, L, seed, n, hits)
    assert st["n_nodes"] == 1 and st["bvh_depth"] == 1 and st["staged_nodes"] == 1, st
    q_staged = tr.texel_sums()
    info = _every_texel(tr, sc, L, seed, n, hits)
    assert info["lit"] == 1 and info["diverged"] <= 1e-3 * n, info
    ref = oracle.forward(sc, L, seed, n, hits, counts=True)
    assert st["segments_forward"] == ref["segments"]
    tr.set_launch(0, 0, 0)
    try:
        tr.trace_forward(seed, n, hits)
        assert tr.stats()["staged_nodes"] == 0
        assert np.array_equal(tr.texel_sums(), q_staged)
        target = np.full(sc.n_texels, 0.5 * float(E[0]), np.float32)
        g = _adjoint_case(tr, sc, L, target, n, hits, seed + 1)
        assert np.all(np.abs(g[0, [0, 1, 2, 5]]) > 0)
    finally:
        tr.set_launch(0, 0, 72 * 1024)


def test_fixed_point_sums_identical_across_launch_shapes(tr):
    sc, L = scenes.office(seed=0, pitch=0.1), scenes.office_lights(0)
    tr.upload_scene(sc)
    tr.set_lights(L)
    ref = None
    kinds = set()
    # nodes through L1 (the office BVH takes 55 KiB), nodes staged, nodes and
    # triangles staged
    for threads, bps, smem, tris in [(256, 0, 48 * 1024, 0), (128, 0, 224, 0), (64, 1, 16 * 1024, 0),
                                     (256, 2, 100 * 1024, 0), (256, 2, 100 * 1024, 200 * 1024),
                                     (0, 0, 72 * 1024, 200 * 1024), (0, 0, 72 * 1024, 0), (32, 3, 224 * 7, 0)]:
        tr.set_launch(threads, bps, smem)
        tr.set_tri_staging(tris)
        tr.trace_forward(5, 1 << 16, 5)
        st = tr.stats()
        kinds.add((st["staged_nodes"] > 0, st["staged_triangles"] > 0))
        q = tr.texel_sums()
        if ref is None:
            ref = q
            assert q.sum() > 0
        else:
            assert np.array_equal(q, ref), (threads, bps, smem, tris)
    assert kinds == {(False, False), (True, False), (True, True)}
    tr.set_tri_staging(200 * 1024)
    tr.set_launch(256, 0, 48 * 1024)
    tr.trace_forward(5, 1 << 16, 5)
    assert np.array_equal(tr.texel_sums(), ref)


def test_gradients_identical_across_launch_shapes(tr):
    # exact 128-bit gradient sums: every launch shape gives the same bits,
    # the returned doubles are the library's one rounding of those sums, and
    # the scale G makes the largest weight times the largest flux constant
    # a number in [1, 2)
    sc, L = scenes.office(seed=0, pitch=0.1), scenes.office_lights(0)
    tr.upload_scene(sc)
    tr.set_lights(L)
    w = scenes.random_weights(sc.n_texels, seed=8)
    tr.set_adjoint_weights(w)
    ref = None
    for threads, bps, smem, tris in [(0, 0, 72 * 1024, 200 * 1024), (0, 0, 72 * 1024, 0), (256, 0, 48 * 1024, 0),
                                     (128, 0, 224, 0), (64, 1, 16 * 1024, 0), (256, 2, 100 * 1024, 200 * 1024),
                                     (32, 3, 224 * 7, 0)]:
        tr.set_launch(threads, bps, smem)
        tr.set_tri_staging(tris)
        g = tr.trace_adjoint(7, 1 << 16, 5)
        if ref is None:
            ref = g
            assert np.all(np.abs(g) > 0)
        else:
            assert np.array_equal(g, ref), (threads, bps, smem, tris)
    tr.set_tri_staging(200 * 1024)
    f, G = tr.gradient_fixed()
    assert np.array_equal(gradient_from_fixed(f, G), ref)
    sizes = parity.light_sizes(1 << 16, L.shape[0])
    I = 0.5 * L[:, 6] ** 2
    omega = 2 * np.pi * (1 - np.cos(L[:, 8]))
    t0 = float(np.max(np.abs(w))) * float(np.max(I * omega / sizes))
    assert G == 2.0 ** np.round(np.log2(G)) and 0.99 <= t0 * G < 2.01, (G, t0)
    tr.set_launch(0, 0, 72 * 1024)


def test_launch_shape_arguments(tr):
    # 0 selects the default (the bound of the kernel the BVH selects: 1024
    # threads, staged or through L1 / as many blocks as fit /
    # no staged nodes), a negative argument keeps the current value
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sc, L = scenes.office(seed=0, pitch=0.1), scenes.office_lights(0)
    tr.upload_scene(sc)
    tr.set_lights(L)

    def shape():
        tr.trace_forward(5, 1 << 14, 5)
        st = tr.stats()
        return st["grid_blocks"], st["block_threads"], st["staged_nodes"]

    tr.set_launch(128, 2, 0)
    assert shape() == (2 * sms, 128, 0)
    tr.set_launch(-1, -1, 200 * 1024)
    assert shape() == (2 * sms, 128, tr.stats()["n_nodes"])
    tr.set_launch(0, 0, -1)
    g, t, staged = shape()
    assert t == 1024 and g % sms == 0 and staged > 0
    # the triangles follow the staged nodes while both fit the budget
    n_tri = tr.stats()["n_triangles"]
    assert tr.stats()["staged_triangles"] == n_tri
    need = staged * 240 + (staged + 3) // 4 * 16 + (n_tri * 52 + 15) // 16 * 16
    tr.set_tri_staging(need - 16)
    assert shape() == (g, t, staged) and tr.stats()["staged_triangles"] == 0
    tr.set_tri_staging(need)
    assert shape() == (g, t, staged) and tr.stats()["staged_triangles"] == n_tri
    # smaller blocks: the triangles would cost resident blocks, so only the
    # nodes are staged
    tr.set_launch(256, 0, -1)
    g2, t2, staged2 = shape()
    assert t2 == 256 and staged2 == staged and g2 >= 2 * sms and tr.stats()["staged_triangles"] == 0
    tr.set_launch(256, 1, -1)
    assert shape() == (sms, 256, staged) and tr.stats()["staged_triangles"] == n_tri
    tr.set_launch(0, 0, -1)
    with pytest.raises(RuntimeError, match="max_bytes"):
        tr.set_tri_staging(221 * 1024)
    with pytest.raises(RuntimeError, match="max_bytes"):
        tr.set_tri_staging(-1)
    tr.set_tri_staging(200 * 1024)
    tr.set_launch(0, 0, 0)
    g, t, staged = shape()
    assert t == 1024 and g % sms == 0 and staged == 0
    # blocks beyond 1024 threads or not a multiple of 32 are refused on the
    # host, before any launch
    for bad in (1056, 100):
        with pytest.raises(RuntimeError, match="multiple of 32"):
            tr.set_launch(bad, 0, 0)
    tr.set_launch(512, 0, 0)
    assert shape()[1:] == (512, 0)
    tr.set_launch(1024, 0, 200 * 1024)
    assert shape() == (sms, 1024, tr.stats()["n_nodes"])
    tr.set_launch(256, 0, 48 * 1024)


def _cornell_target(sc, lights):
    Lt = scenes.perturb_lights(lights, seed=1, pos_sigma=0.05)
    return oracle.forward(sc, Lt, 101, 1 << 16, 3)["E"].astype(np.float32)


def test_loss_matches_oracle(tr):
    sc, L = scenes.cornell_box(res=32), scenes.cornell_lights()
    target = _cornell_target(sc, L)
    alpha = np.random.default_rng(3).uniform(0.5, 1.5, sc.n_texels).astype(np.float32)
    n, hits, seed = 1 << 20, 3, 2
    tr.upload_scene(sc)
    tr.set_lights(L)
    tr.set_target(target, alpha)
    tr.trace_forward(seed, n, hits)
    O = tr.loss()
    ref = oracle.forward(sc, L, seed, n, hits)
    O_ref, _ = oracle.loss(sc, ref["E"], target, alpha)
    assert abs(O - O_ref) <= 1e-4 * O_ref, (O, O_ref)


def _adjoint_case(tr, sc, L, target, n, hits, seed, term_tol=1e-2):
    """GPU forward + loss + adjoint as a user runs them, then the same adjoint
    on both sides from identical weights (the oracle's, rounded to float)."""
    tr.upload_scene(sc)
    tr.set_lights(L)
    tr.set_target(target)
    tr.trace_forward(seed, n, hits)
    tr.loss()
    g_own = tr.trace_adjoint(seed, n, hits)
    assert np.array_equal(g_own, tr.trace_adjoint(seed, n, hits))     # deterministic rerun
    ref = oracle.forward(sc, L, seed, n, hits)
    _, w = oracle.loss(sc, ref["E"], target, np.ones(sc.n_texels))
    w32 = w.astype(np.float32)
    tr.set_adjoint_weights(w32)
    g = tr.trace_adjoint(seed, n, hits)
    g_ref, _ = oracle.adjoint(sc, L, seed, n, hits, w32.astype(np.float64))
    parity.check_gradient(tr, sc, L, seed, n, hits, w32.astype(np.float64), g, g_ref, term_tol=term_tol)
    # with its own weights the GPU gradient still tracks the oracle's
    assert np.abs(g_own - g_ref).max() <= 1e-2 * np.abs(g_ref).max()
    return g


def test_adjoint_matches_oracle_cornell_point(tr):
    sc, L = scenes.cornell_box(res=32), scenes.cornell_lights()
    g = _adjoint_case(tr, sc, L, _cornell_target(sc, L), 1 << 18, 3, 2)
    assert np.all(g[:, [3, 4, 6, 7]] == 0)


def test_adjoint_matches_oracle_office_spots(tr):
    sc, L = scenes.office(seed=0, pitch=0.1), scenes.office_lights(0)
    Lt = scenes.perturb_lights(L, seed=2, pos_sigma=0.3, angle_sigma=0.1, intensity_range=(0.7, 1.3),
                               theta_in_delta=np.radians(5))
    target = oracle.forward(sc, Lt, 77, 1 << 16, 5)["E"].astype(np.float32)
    g = _adjoint_case(tr, sc, L, target, 1 << 16, 5, 4)
    assert np.all(np.abs(g) > 0)


def test_adjoint_with_injected_weights(tr):
    sc = scenes.cornell_box(res=16)
    L = scenes.make_lights([scenes.spot_light((0.45, 0.5, 0.92), 0.3, -1.35, 1.0, 0.45, 0.9),
                            scenes.point_light((0.2, 0.7, 0.5), 0.5)])
    w = scenes.random_weights(sc.n_texels, seed=5)
    n, hits, seed = 100_000, 3, 9
    tr.upload_scene(sc)
    tr.set_lights(L)
    tr.set_adjoint_weights(w)
    g = tr.trace_adjoint(seed, n, hits)
    g_ref, _ = oracle.adjoint(sc, L, seed, n, hits, w.astype(np.float64))
    parity.check_gradient(tr, sc, L, seed, n, hits, w.astype(np.float64), g, g_ref)


def test_deep_bvh_staged_and_through_l1(tr):
    # A BVH of more than 8 levels that fits in shared memory: the staged
    # kernel with two words of pending masks. Every ray from the apex light
    # descends the whole chain of nested strips. Irradiance and gradients
    # must match the oracle, and the kernel that reads nodes through L1 must
    # give the same integer sums.
    sc = scenes.nested_shelf()
    L = scenes.make_lights([scenes.point_light(scenes.NESTED_SHELF_APEX, 1.0)])
    n, hits, seed = 1 << 19, 3, 4
    tr.set_launch(0, 0, 72 * 1024)
    E, st = _forward(tr, sc, L, seed, n, hits)
    assert st["bvh_depth"] > 8 and st["staged_nodes"] == st["n_nodes"] > 0, st
    assert st["block_threads"] == 1024
    q_staged = tr.texel_sums()
    ref = oracle.forward(sc, L, seed, n, hits, counts=True)
    assert _check_irradiance(sc, E, ref, min_count=1000) > 300
    # the room is closed: every photon makes exactly `hits` segments
    assert st["segments_forward"] == n * hits == ref["segments"]
    tr.set_launch(0, 0, 0)
    tr.trace_forward(seed, n, hits)
    st = tr.stats()
    assert st["staged_nodes"] == 0 and st["block_threads"] == 1024
    assert np.array_equal(tr.texel_sums(), q_staged)
    tr.set_launch(0, 0, 72 * 1024)
    Lt = L.copy()
    Lt[0, 1:4] += (0.2, -0.1, 0.3)
    target = oracle.forward(sc, Lt, 77, 1 << 16, hits)["E"].astype(np.float32)
    g = _adjoint_case(tr, sc, L, target, 1 << 16, hits, 5)
    assert np.all(np.abs(g[0, [0, 1, 2, 5]]) > 0)


def test_call_order_and_argument_errors():
    t = Tracer(0)
    try:
        with pytest.raises(LtError):
            t.trace_forward(1, 100, 3)               # no scene
        t.upload_scene(scenes.cornell_box(res=4))
        with pytest.raises(LtError):
            t.trace_forward(1, 100, 3)               # no lights
        t.set_lights(scenes.cornell_lights())
        with pytest.raises(LtError):
            t.trace_forward(1, 100, 0)               # max_hits out of range
        with pytest.raises(LtError):
            t.trace_forward(1, 100, 3, 50, 101)      # range beyond the budget
        with pytest.raises(LtError):
            t.loss()                                 # no forward pass
        t.trace_forward(1, 100, 3)
        with pytest.raises(LtError):
            t.loss()                                 # no target
        with pytest.raises(LtError):
            t.trace_adjoint(1, 100, 3)               # no weights
        with pytest.raises(LtError):
            t.set_lights(scenes.make_lights([scenes.spot_light((0, 0, 0), 0, 0, 1, 0.5, 0.5)]))  # empty soft edge
    finally:
        t.close()
