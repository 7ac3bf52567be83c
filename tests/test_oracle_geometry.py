"""Pins for the oracle's ray casting and texel lookup.

The reference is an independent double-precision brute force (the
Moller-Trumbore test, written here with numpy), and analytic plane hits."""
import numpy as np

import oracle
from paper_2310_02043_gb300 import scenes


def _mt_all(xyz, o, d):
    """Moller-Trumbore in float64 for one ray against all triangles:
    returns t (inf on a miss) and barycentrics (1-b1-b2, b1, b2)."""
    v0, v1, v2 = xyz[:, 0].astype(np.float64), xyz[:, 1].astype(np.float64), xyz[:, 2].astype(np.float64)
    e1, e2 = v1 - v0, v2 - v0
    p = np.cross(d, e2)
    det = np.einsum("ij,ij->i", e1, p)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / det
        s = o - v0
        b1 = np.einsum("ij,ij->i", s, p) * inv
        q = np.cross(s, e1)
        b2 = (q @ d) * inv
        t = np.einsum("ij,ij->i", e2, q) * inv
    ok = (np.abs(det) > 1e-14) & (b1 >= 0) & (b2 >= 0) & (b1 + b2 <= 1) & (t > 0)
    t = np.where(ok, t, np.inf)
    return t, np.stack([1 - b1 - b2, b1, b2], 1)


def test_closest_hit_matches_fp64_brute_force():
    sc = scenes.random_triangles(40, seed=3)
    o, d = scenes.random_rays(3000, seed=4)
    tri, t, b = oracle.closest_hits(sc, o, d)
    xyz = sc.xyz
    checked = 0
    for i in range(len(o)):
        tt, bb = _mt_all(xyz, o[i], d[i])
        order = np.argsort(tt)
        best = order[0]
        if not np.isfinite(tt[best]):
            continue        # misses are checked separately
        # skip near-ties between two surfaces and hits within 1e-5 of an edge
        near_tie = len(order) > 1 and np.isfinite(tt[order[1]]) and tt[order[1]] - tt[best] < 1e-5 * tt[best]
        near_edge = bb[best].min() < 1e-5
        if near_tie or near_edge:
            continue
        assert tri[i] == best, (i, tri[i], best)
        assert abs(t[i] - tt[best]) <= 1e-5 * (tt[best] + 1.0)   # float error scales with the scene
        np.testing.assert_allclose(b[i], bb[best], atol=1e-5)
        checked += 1
    assert checked > 500


def test_misses_far_from_edges_are_misses():
    sc = scenes.random_triangles(40, seed=5)
    o, d = scenes.random_rays(2000, seed=6)
    tri, t, b = oracle.closest_hits(sc, o, d)
    for i in range(len(o)):
        tt, bb = _mt_all(sc.xyz, o[i], d[i])
        if not np.isfinite(tt).any():
            # no fp64 hit: the float test may only report one on an edge
            if tri[i] >= 0:
                assert b[i].min() < 1e-5


def test_watertight_on_shared_diagonal():
    # Rays aimed at points on the shared diagonal of a quad never slip through.
    sc = scenes.plane(half=1.0, res=4)
    s = np.linspace(-0.999, 0.999, 501)
    target = np.stack([s, s, np.zeros_like(s)], 1)
    rng = np.random.default_rng(0)
    o = target + np.stack([rng.uniform(-0.5, 0.5, len(s)), rng.uniform(-0.5, 0.5, len(s)), np.full(len(s), 1.0)], 1)
    d = target - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    tri, t, b = oracle.closest_hits(sc, o, d)
    assert np.all(tri >= 0)


def test_skip_tile_excludes_the_tile_left():
    sc = scenes.closed_cube(size=1.0, res=2)
    o = np.array([[0.5, 0.5, -1e-4]])     # a hit point rounded just below the floor
    d = np.array([[0.0, 0.0, 1.0]])
    tri, t, _ = oracle.closest_hits(sc, o, d, skip_tile=-1)
    floor_tile = sc.tile[tri[0]]
    assert abs(t[0] - 1e-4) < 1e-7         # not skipped: the floor again
    tri2, t2, _ = oracle.closest_hits(sc, o, d, skip_tile=int(floor_tile))
    assert sc.tile[tri2[0]] != floor_tile and abs(t2[0] - 1.0001) < 1e-6   # the ceiling


def test_texels_of_direct_hits_match_analytic_plane_hits():
    # Point light above a 16x16-texel plane, one hit per photon: the texel the
    # oracle deposits into equals the texel of the analytic ray/plane hit.
    half, res, h = 1.0, 16, 0.7
    sc = scenes.plane(half=half, res=res)
    pos = np.array([0.1, -0.2, h])
    lights = scenes.make_lights([scenes.point_light(pos, 1.0)])
    n = 4000
    tri, tex = oracle.paths(sc, lights, seed=9, n_photons=n, max_hits=1, begin=0, count=n)
    agree = 0
    for k in range(n):
        w, phi, a = oracle.emit(lights[0], n, 9, k)
        if w[2] >= 0:
            assert tri[k, 0] == -1
            continue
        t = -h / w[2]
        x = pos + t * w
        u, v = (x[0] + half) / (2 * half), (x[1] + half) / (2 * half)
        if not (0 < u < 1 and 0 < v < 1):
            assert tri[k, 0] == -1 or min(abs(u), abs(1 - u), abs(v), abs(1 - v)) < 1e-5
            continue
        fu, fv = u * res, v * res
        if min(abs(fu - round(fu)), abs(fv - round(fv))) < 1e-4:
            continue
        assert tex[k, 0] == int(fu) + res * int(fv)
        agree += 1
    assert agree > 600
