"""Pins for the oracle's forward pass (Alg. 1, Eq. 7-8) against closed forms.

* emission and bounce sampling distributions (uniform sphere, uniform cone,
  cosine lobe) by Kolmogorov-Smirnov tests;
* energy: in a closed scene nothing escapes, so sum_t A_t E_t equals the
  emitted power times sum_{i<B} rho^i exactly;
* inverse-square law: with one hit, a texel's irradiance is I Omega_t / A_t
  (point light) or the quadrature of I a cos / r^2 (spot);
* interior sphere: cosine-weighted reflection from any point of a sphere lands
  uniformly on it, so the second-hit irradiance is uniform even for an
  off-centre light, and B hits add the geometric series of rho;
* several lights: the budget split and each light's normalisation."""
import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2310_02043_gb300 import scenes
from tests import closed_forms as cf


def test_point_emission_is_uniform_on_the_sphere():
    light = scenes.make_lights([scenes.point_light((0, 0, 0), 2.0)])[0]
    n = 4000
    W = np.array([oracle.emit(light, n, 5, k)[0] for k in range(n)])
    np.testing.assert_allclose(np.linalg.norm(W, axis=1), 1.0, atol=1e-12)
    assert stats.kstest(W[:, 2], "uniform", args=(-1, 2)).pvalue > 1e-3
    az = np.arctan2(W[:, 1], W[:, 0])
    assert stats.kstest(az, "uniform", args=(-np.pi, 2 * np.pi)).pvalue > 1e-3
    _, phi, a = oracle.emit(light, n, 5, 0)
    assert phi == pytest.approx(2.0 * 4 * np.pi / n, rel=1e-14) and a == 1.0


def test_spot_emission_is_uniform_in_the_outer_cone():
    yaw, pitch, th_in, th_out = 0.7, -1.1, 0.3, 0.8
    light = scenes.make_lights([scenes.spot_light((0, 0, 0), yaw, pitch, 3.0, th_in, th_out)])[0]
    axis = cf.spot_axis(yaw, pitch)
    n = 4000
    rows = [oracle.emit(light, n, 8, k) for k in range(n)]
    W = np.array([r[0] for r in rows])
    c = W @ axis
    co, ci = np.cos(th_out), np.cos(th_in)
    assert c.min() >= co - 1e-12
    assert stats.kstest(c, "uniform", args=(co, 1 - co)).pvalue > 1e-3
    # azimuth about the axis is uniform
    ref = np.cross(axis, [1.0, 0.0, 0.0]); ref /= np.linalg.norm(ref)
    ref2 = np.cross(axis, ref)
    az = np.arctan2(W @ ref2, W @ ref)
    assert stats.kstest(az, "uniform", args=(-np.pi, 2 * np.pi)).pvalue > 1e-3
    # flux: I * 2 pi (1 - cos th_out) * a(theta) / N with the falloff of Eq. S.11
    phi = np.array([r[1] for r in rows])
    a = cf.spot_quadratic_falloff(c, ci, co)
    np.testing.assert_allclose(phi, 3.0 * 2 * np.pi * (1 - co) * a / n, rtol=1e-9, atol=1e-15)


def test_cosine_directions_follow_the_cosine_lobe():
    rng = np.random.default_rng(1)
    for _ in range(4):
        nrm = rng.normal(size=3); nrm /= np.linalg.norm(nrm)
        if rng.uniform() < 0.3:
            nrm = np.array([0.0, 0.0, -1.0]) if rng.uniform() < 0.5 else np.array([1.0, 0.0, 0.0])
        u = rng.uniform(size=(3000, 2))
        W = np.array([oracle.cosine_dir(nrm, a, b) for a, b in u])
        np.testing.assert_allclose(np.linalg.norm(W, axis=1), 1.0, atol=1e-12)
        c = W @ nrm
        assert c.min() > 0
        # cosine-weighted: cos^2(theta) is uniform on [0, 1]
        assert stats.kstest(c * c, "uniform").pvalue > 1e-3


def test_energy_closed_cube_point_light_is_exact():
    rho, B, I = 0.6, 4, 1.7
    sc = scenes.closed_cube(size=1.0, res=6, albedo=rho)
    L = scenes.make_lights([scenes.point_light((0.31, 0.62, 0.44), I)])
    r = oracle.forward(sc, L, seed=3, n_photons=20000, max_hits=B)
    A = oracle.texel_areas(sc)
    rho32 = float(np.float32(rho))        # albedo is stored as float32
    expect = I * 4 * np.pi * sum(rho32 ** i for i in range(B))
    assert np.sum(A * r["E"]) == pytest.approx(expect, rel=1e-12)
    assert r["segments"] == 20000 * B and r["deposits"] == 20000 * B


def test_path_record_flux_per_hit():
    # The path record's per-hit flux (Eq. 7): in a closed cube with a point
    # light every ray carries I 4 pi / N, and hit i of every photon carries
    # rho^(i-1) of it, so the flux of hit i summed over photons is
    # 4 pi I rho^(i-1) exactly; with per-face albedo, hit i + 1 carries hit
    # i's flux times the albedo of the face hit i landed on.
    rho, B, I, n = 0.6, 4, 1.7, 5000
    sc = scenes.closed_cube(size=1.0, res=6, albedo=rho)
    L = scenes.make_lights([scenes.point_light((0.31, 0.62, 0.44), I)])
    tri, tex, phi = oracle.paths(sc, L, 3, n, B, 0, n, flux=True)
    assert np.all(tri >= 0)
    rho32 = float(np.float32(rho))
    for i in range(B):
        assert phi[:, i].sum() == pytest.approx(4 * np.pi * I * rho32 ** i, rel=1e-12)
    rho_face = np.array([0.9, 0.1, 0.3, 0.6, 0.45, 0.75], np.float32)
    sc.albedo = np.ascontiguousarray(rho_face[sc.tile])
    tri, tex, phi = oracle.paths(sc, L, 3, n, B, 0, n, flux=True)
    ratio = phi[:, 1:] / phi[:, :-1]
    np.testing.assert_allclose(ratio, rho_face[sc.tile[tri[:, :-1]]].astype(np.float64), rtol=1e-13)
    # the record's deposits are the forward pass's (Eq. 8)
    A = oracle.texel_areas(sc)
    E = np.bincount(tex.ravel(), weights=phi.ravel(), minlength=sc.n_texels) / A
    np.testing.assert_allclose(E, oracle.forward(sc, L, 3, n, B)["E"], rtol=1e-12, atol=0)


def test_bounce_flux_uses_the_albedo_of_the_surface_left():
    # Eq. 7 with a Lambertian f and cosine sampling: Phi_{i+1} = rho(x_i) Phi_i.
    # With per-face albedo, the second-hit energy equals sum_f rho_f times the
    # first-hit energy landing on face f -- exactly, for the same seed.
    sc = scenes.closed_cube(size=1.0, res=3, albedo=0.5)
    rho_face = np.array([0.9, 0.1, 0.3, 0.6, 0.45, 0.75], np.float32)
    sc.albedo = np.ascontiguousarray(rho_face[sc.tile])
    L = scenes.make_lights([scenes.point_light((0.3, 0.6, 0.45), 1.0)])
    n = 1 << 14
    r1 = oracle.forward(sc, L, 6, n, 1)
    r2 = oracle.forward(sc, L, 6, n, 2)
    A = oracle.texel_areas(sc)
    per_texel_tile = np.repeat(np.arange(6), 9)
    e1_face = np.bincount(per_texel_tile, weights=A * r1["E"], minlength=6)
    second = np.sum(A * (r2["E"] - r1["E"]))
    assert second == pytest.approx(float(np.sum(rho_face.astype(np.float64) * e1_face)), rel=1e-11)


def test_energy_closed_cube_spot_matches_cone_integral():
    # E[sum_r Phi_r] = I * 2 pi * int_{co}^{1} a(c) dc = I 2 pi ((1 - ci) + (ci - co) / 3)
    rho, B, I, th_in, th_out = 0.5, 2, 2.0, 0.35, 0.9
    sc = scenes.closed_cube(size=1.0, res=4, albedo=rho)
    L = scenes.make_lights([scenes.spot_light((0.5, 0.5, 0.8), 0.2, -1.3, I, th_in, th_out)])
    n = 1 << 16
    r = oracle.forward(sc, L, seed=4, n_photons=n, max_hits=B)
    A = oracle.texel_areas(sc)
    emitted = np.sum(A * r["E"]) / (1 + float(np.float32(rho)))
    ci, co = np.cos(th_in), np.cos(th_out)
    expect = I * 2 * np.pi * ((1 - ci) + (ci - co) / 3)
    # per-ray flux I Omega a / N with a(c) of c ~ U[co, 1]: variance from E[a^2]
    Ea2 = ((1 - ci) + (ci - co) / 5) / (1 - co)
    Ea = ((1 - ci) + (ci - co) / 3) / (1 - co)
    sigma = I * 2 * np.pi * (1 - co) * np.sqrt((Ea2 - Ea * Ea) / n)
    assert abs(emitted - expect) < 5 * sigma


def test_point_light_irradiance_on_plane_is_inverse_square():
    half, res, I = 1.0, 12, 1.3
    pos = (0.15, -0.1, 0.6)
    sc = scenes.plane(half=half, res=res)
    L = scenes.make_lights([scenes.point_light(pos, I)])
    n = 1 << 20
    r = oracle.forward(sc, L, seed=21, n_photons=n, max_hits=1, counts=True)
    A = (2 * half / res) ** 2
    omega = cf.plane_texel_solid_angles(half, res, np.array(pos))
    expect = I * omega / A
    phi = I * 4 * np.pi / n
    p = omega / (4 * np.pi)
    sigma = phi / A * np.sqrt(n * p * (1 - p))
    z = (r["E"] - expect) / sigma
    assert np.max(np.abs(z)) < 5.0
    assert abs(np.mean(z * z) - 1.0) < 0.35          # chi-square / dof
    # every deposit carries the same flux
    np.testing.assert_allclose(r["E"] * A, r["count"] * phi, rtol=1e-12)


def test_spot_irradiance_on_plane_matches_quadrature():
    half, res = 1.5, 10
    light = scenes.spot_light((0.1, 0.2, 1.0), 0.4, -np.pi / 2 + 0.25, 2.0, 0.25, 0.7)
    sc = scenes.plane(half=half, res=res)
    L = scenes.make_lights([light])
    n = 1 << 20
    r = oracle.forward(sc, L, seed=22, n_photons=n, max_hits=1)
    A = (2 * half / res) ** 2
    expect = cf.plane_texel_spot_flux(half, res, np.array(light), sub=8, order=6) / A
    phi_max = 2.0 * 2 * np.pi * (1 - np.cos(0.7)) / n
    sigma = np.sqrt(phi_max * np.maximum(expect, 1e-30) / A) + 1e-12
    z = (r["E"] - expect) / sigma
    assert np.max(np.abs(z)) < 5.0
    assert np.sum(r["E"]) == pytest.approx(np.sum(expect), rel=5e-3)


def test_sphere_direct_is_solid_angle_and_second_hit_is_uniform():
    R, rho, I = 1.0, 0.5, 1.0
    sc = scenes.icosphere(radius=R, subdiv=3, albedo=rho)
    pos = np.array([0.3, 0.2, -0.35])
    L = scenes.make_lights([scenes.point_light(pos, I)])
    n = 1 << 21
    r1 = oracle.forward(sc, L, seed=5, n_photons=n, max_hits=1, counts=True)
    r2 = oracle.forward(sc, L, seed=5, n_photons=n, max_hits=2, counts=True)
    A = sc.tile_area
    phi = I * 4 * np.pi / n
    # direct: E_f = I Omega_f / A_f, exact up to Monte Carlo noise
    omega = np.array([cf.triangle_solid_angle(*sc.xyz[f].astype(np.float64), pos) for f in range(sc.n_tri)])
    assert np.sum(omega) == pytest.approx(4 * np.pi, rel=1e-9)
    p = omega / (4 * np.pi)
    z1 = (r1["E"] - I * omega / A) / (phi / A * np.sqrt(n * p * (1 - p)))
    assert np.max(np.abs(z1)) < 5.0 and abs(np.mean(z1 * z1) - 1) < 0.3
    # second hit: same seed, so the difference is exactly the second deposits
    E2 = r2["E"] - r1["E"]
    c2 = r2["count"] - r1["count"]
    total = I * 4 * np.pi * float(np.float32(rho))
    assert np.sum(A * E2) == pytest.approx(total, rel=1e-10)
    mean = total / np.sum(A)
    sigma = rho * phi * np.sqrt(np.maximum(c2, 1)) / A
    chi2 = np.mean(((E2 - mean) / sigma) ** 2)
    assert 0.8 < chi2 < 1.3, chi2


def test_sphere_interreflection_is_the_geometric_series():
    """Inside a diffuse sphere every reflected photon lands uniformly per unit
    area, whatever its origin, so with B hits each texel holds its direct
    irradiance plus (4 pi I / A_sphere) (rho + ... + rho^(B-1)), which tends to
    the direct term plus rho / (1 - rho) of the mean: the 1 / (1 - rho)
    interreflection of Eq. 7 applied at every hit.

    A bounce ray starts at the hit point without an offset, and a hit point
    computed from a float distance can land a rounding error outside the
    surface; near an edge, a grazing bounce towards the neighbouring face can
    then leave the closed mesh (about one segment in a million here). The
    energy identity is checked exactly against the hits each photon made."""
    R, rho, I, B = 1.0, 0.5, 1.0, 12
    sc = scenes.icosphere(radius=R, subdiv=3, albedo=rho)
    pos = np.array([-0.25, 0.4, 0.1])
    L = scenes.make_lights([scenes.point_light(pos, I)])
    n = 1 << 18
    r1 = oracle.forward(sc, L, seed=9, n_photons=n, max_hits=1)
    rB = oracle.forward(sc, L, seed=9, n_photons=n, max_hits=B)
    tri, _ = oracle.paths(sc, L, 9, n, B, 0, n)
    hits = np.sum(tri >= 0, axis=1)
    assert np.all(tri[np.arange(B)[None, :] >= hits[:, None]] < 0)      # a path ends at its first miss
    assert np.all(hits >= 1) and np.sum(B - hits) <= 1e-5 * n * B       # escapes are rare
    A = sc.tile_area
    phi = I * 4 * np.pi / n
    Eind = rB["E"] - r1["E"]
    geo = np.concatenate([[0.0], np.cumsum(rho ** np.arange(1, B))])      # rho + ... + rho^(h-1)
    assert np.sum(A * Eind) == pytest.approx(phi * np.sum(geo[hits - 1]), rel=1e-10)
    series = geo[B - 1]
    mean = I * 4 * np.pi / np.sum(A) * series
    assert mean * (1 - rho) / rho == pytest.approx(I * 4 * np.pi / np.sum(A), rel=1e-3)   # the 1/(1-rho) limit
    # per texel: a photon's hits after the first are nearly independent
    # uniform draws, one deposit of rho^i phi each
    p = A / np.sum(A)
    sigma = phi * np.sqrt(n * p * np.sum(rho ** (2.0 * np.arange(1, B)))) / A
    chi2 = np.mean(((Eind - mean) / sigma) ** 2)
    assert 0.75 < chi2 < 1.35, chi2


def test_two_lights_split_the_budget_and_superpose():
    """With L lights a budget of N photons is split evenly, the first N mod L
    lights taking one extra, and each photon carries I Omega / N_l of its own
    light: irradiance is the sum of the lights' closed forms, and light 0's
    photon range reproduces light 0 traced alone with N_0 photons exactly."""
    half, res = 1.5, 10
    point = scenes.point_light((0.15, -0.1, 0.6), 1.3)
    spot = scenes.spot_light((0.1, 0.2, 1.0), 0.4, -np.pi / 2 + 0.25, 2.0, 0.25, 0.7)
    sc = scenes.plane(half=half, res=res)
    L = scenes.make_lights([point, spot])
    n = (1 << 20) + 1
    n0, n1 = (n + 1) // 2, n // 2
    r = oracle.forward(sc, L, seed=23, n_photons=n, max_hits=1)
    A = (2 * half / res) ** 2
    omega = cf.plane_texel_solid_angles(half, res, np.array(point[1:4]))
    e_point = 1.3 * omega / A
    e_spot = cf.plane_texel_spot_flux(half, res, np.array(spot), sub=8, order=6) / A
    phi_p = 1.3 * 4 * np.pi / n0
    phi_s = 2.0 * 2 * np.pi * (1 - np.cos(0.7)) / n1
    p = omega / (4 * np.pi)
    var = (phi_p / A) ** 2 * n0 * p * (1 - p) + phi_s * np.maximum(e_spot, 1e-30) / A
    z = (r["E"] - e_point - e_spot) / np.sqrt(var)
    assert np.max(np.abs(z)) < 5.0
    # light 0 owns photons [0, n0) and normalises by its own count
    alone = oracle.forward(sc, scenes.make_lights([point]), seed=23, n_photons=n0, max_hits=1)
    part = oracle.forward(sc, L, seed=23, n_photons=n, max_hits=1, begin=0, end=n0)
    assert np.array_equal(part["E"], alone["E"])
    rest = oracle.forward(sc, L, seed=23, n_photons=n, max_hits=1, begin=n0, end=n)
    np.testing.assert_allclose(part["E"] + rest["E"], r["E"], rtol=1e-12)
    w = np.random.default_rng(3).normal(size=sc.n_texels)
    g_part, _ = oracle.adjoint(sc, L, 23, n, 1, w, begin=0, end=n0)
    g_alone, _ = oracle.adjoint(sc, scenes.make_lights([point]), 23, n0, 1, w)
    assert np.array_equal(g_part[0], g_alone[0]) and not np.any(g_part[1])
