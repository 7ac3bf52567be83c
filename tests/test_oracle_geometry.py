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


def _mt_raw(xyz, o, d):
    """Moller-Trumbore in float64 without the inside test: t and the three
    barycentrics of the ray's crossing with every triangle's plane."""
    v0, v1, v2 = xyz[:, 0].astype(np.float64), xyz[:, 1].astype(np.float64), xyz[:, 2].astype(np.float64)
    e1, e2 = v1 - v0, v2 - v0
    p = np.cross(d, e2)
    det = np.einsum("ij,ij->i", e1, p)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / det
        s = o - v0
        b1 = np.einsum("ij,ij->i", s, p) * inv
        b2 = (np.cross(s, e1) @ d) * inv
        t = np.einsum("ij,ij->i", e2, np.cross(s, e1)) * inv
    return t, np.stack([1 - b1 - b2, b1, b2], 1)


def test_near_edge_hits_are_consistent():
    # The rays the brute-force comparison above leaves out, made on purpose:
    # each aims at a point within 1e-5 (in barycentrics) of an edge or a
    # corner of a triangle of the soup. On every ray the oracle's hit lies on
    # a triangle that the exact test hits or misses by a rounding margin, at
    # that triangle's exact distance, and never behind a triangle that the ray
    # crosses clearly inside.
    sc = scenes.random_triangles(40, seed=3)
    rng = np.random.default_rng(13)
    n = 6000
    k = rng.integers(0, sc.n_tri, n)
    bary = np.empty((n, 3))
    bary[:, 0] = rng.uniform(-1e-5, 1e-5, n)                 # across the edge opposite corner 0
    bary[:, 1] = rng.uniform(0, 1, n) * (1 - bary[:, 0])
    corner = rng.uniform(0, 1, n) < 0.2                      # a fifth of them next to corner 1
    bary[corner, 1] = 1 - rng.uniform(-1e-5, 2e-5, corner.sum())
    bary[:, 2] = 1 - bary[:, 0] - bary[:, 1]
    roll = rng.integers(0, 3, n)                             # which edge
    bary = np.stack([np.roll(bary[i], roll[i]) for i in range(n)])
    xyz = sc.xyz.astype(np.float64)
    target = np.einsum("ij,ijk->ik", bary, xyz[k])
    o = target + rng.normal(0, 1, (n, 3))
    d = target - o
    dist = np.linalg.norm(d, axis=1)
    d /= dist[:, None]
    tri, t, _ = oracle.closest_hits(sc, o, d)
    normal = np.cross(xyz[:, 1] - xyz[:, 0], xyz[:, 2] - xyz[:, 0])
    normal /= np.linalg.norm(normal, axis=1, keepdims=True)
    front = np.zeros(n, bool)                # another triangle lies in front of the target
    for i in range(n):
        tt, bb = _mt_raw(sc.xyz, o[i], d[i])
        ok = np.isfinite(tt) & (tt > 0)
        clear = ok & (bb.min(axis=1) > 1e-5)
        loose = ok & (bb.min(axis=1) > -1e-5)
        t_clear = tt[clear].min() if clear.any() else np.inf
        others = loose & (tt < dist[i] * (1 - 1e-4))
        others[k[i]] = False
        front[i] = others.any()
        if tri[i] < 0:
            assert not np.isfinite(t_clear), i
            continue
        j = tri[i]
        assert loose[j], (i, j, bb[j])
        # t moves by the rounding of the ray over the cosine of its incidence
        cos_j = abs(normal[j] @ d[i])
        assert abs(t[i] - tt[j]) <= 1e-5 * (tt[j] + 1.0) / max(cos_j, 1e-3), (i, j, cos_j)
        assert t[i] <= t_clear + 1e-5 * (t_clear + 1.0) / max(cos_j, 1e-3)
    # Where nothing lies in front, the float test decides inside or outside
    # correctly once the target is farther from the aimed-at triangle's edges
    # than the rounding of the ray and the vertices (a few float ulps of the
    # coordinates involved, on both sides of the edge).
    P = xyz[k]
    area2 = np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    opposite = np.stack([np.linalg.norm(P[:, (m + 2) % 3] - P[:, (m + 1) % 3], axis=1) for m in range(3)], 1)
    edge_dist = (bary * (area2[:, None] / opposite)).min(axis=1)   # signed distance to the nearest edge line
    ulp = 2.0 ** -23 * (np.abs(o).max(axis=1) + dist)
    clear_in, clear_out = ~front & (edge_dist > 8 * ulp), ~front & (edge_dist < -8 * ulp)
    assert clear_in.sum() > 200 and clear_out.sum() > 200
    assert np.all(tri[clear_in] == k[clear_in])
    np.testing.assert_allclose(t[clear_in], dist[clear_in], rtol=1e-5)
    assert np.all(tri[clear_out] != k[clear_out])


def _edges(xyz):
    """Vertices and edge midpoints of a triangle mesh (float32 corners), each once."""
    v = xyz.reshape(-1, 3).astype(np.float64)
    e = np.concatenate([(xyz[:, a] + xyz[:, b]) * 0.5 for a, b in ((0, 1), (1, 2), (2, 0))]).astype(np.float64)
    return np.unique(np.concatenate([v, e]), axis=0)


def test_rays_at_vertices_and_edges_of_a_closed_mesh_never_leak():
    # From inside a closed convex mesh, a ray aimed exactly at a vertex (where
    # five or six triangles meet) or at a point of a shared edge leaves the
    # mesh there: it must hit, at the distance of that point.
    rng = np.random.default_rng(11)
    for sc in (scenes.icosphere(radius=1.0, subdiv=2), scenes.closed_cube(size=1.0, res=2)):
        targets = _edges(sc.xyz)
        centre = targets.mean(axis=0)
        for rep in range(3):
            o = centre + rng.uniform(-0.3, 0.3, targets.shape)
            d = targets - o
            dist = np.linalg.norm(d, axis=1)
            d /= dist[:, None]
            tri, t, b = oracle.closest_hits(sc, o, d)
            assert np.all(tri >= 0), f"{sc.name}: {(tri < 0).sum()} of {len(tri)} rays leaked"
            np.testing.assert_allclose(t, dist, rtol=1e-5, atol=1e-6)
            assert b.min() > -1e-5


def test_grazing_rays_hit_the_plane_at_the_analytic_point():
    # Rays that meet the plane z = 0 at a shallow angle (down to 1e-3 rad)
    # hit it where the analytic intersection lies, texel edges included.
    sc = scenes.plane(half=1.0, res=4)
    rng = np.random.default_rng(12)
    n = 2000
    target = np.stack([rng.uniform(-0.95, 0.95, n), rng.uniform(-0.95, 0.95, n), np.zeros(n)], 1)
    target[: n // 4, 0] = 0.0                           # on the shared edge of two quads' texels
    target[n // 4: n // 2, :2] = target[n // 4: n // 2, :1]   # on a quad's diagonal
    elev = 10.0 ** rng.uniform(-3, -1, n)
    az = rng.uniform(0, 2 * np.pi, n)
    d = np.stack([np.cos(az) * np.cos(elev), np.sin(az) * np.cos(elev), -np.sin(elev)], 1)
    dist = 0.05 / np.sin(elev) * rng.uniform(0.5, 1.0, n)      # start 2.5 to 5 cm above the plane
    dist = np.minimum(dist, 0.5)
    o = target - dist[:, None] * d
    tri, t, _ = oracle.closest_hits(sc, o, d)
    assert np.all(tri >= 0)
    hit = o + t[:, None].astype(np.float64) * d
    assert np.max(np.abs(hit[:, :2] - target[:, :2])) < 1e-5
    np.testing.assert_allclose(t, dist, rtol=1e-5, atol=1e-6)
