"""Pins for the oracle's adjoint pass (Alg. 2, Eq. 11-15, S.11-S.12).

* Parameters that leave every path unchanged under a fixed seed (intensity
  p_int, inner cone theta_in) make the same-seed objective a smooth function
  of them; its central finite difference must equal the adjoint gradient,
  through multiple bounces and occlusion (Cornell box).
* For the others (position, yaw/pitch, theta_out) the first hit is held fixed
  (Sec. 4.4.2), which makes the estimator unbiased for the derivative of the
  expected objective when nothing occludes the receiver: one bounce onto a
  plane, adjoint weights injected, compared with a finite difference of the
  closed-form / quadrature expectation.
* A light centred over a symmetric plane with a zero target has no lateral
  gradient; raising it lowers the irradiance, so dO/dz < 0."""
import numpy as np
import pytest

import oracle
from paper_2310_02043_gb300 import scenes
from tests import closed_forms as cf


def _objective(sc, L, seed, n, B, target, alpha):
    E = oracle.forward(sc, L, seed, n, B)["E"]
    return oracle.loss(sc, E, target, alpha)


def _cornell_spot_setup():
    sc = scenes.cornell_box(res=16)
    rho_tile = np.random.default_rng(4).uniform(0.2, 0.9, sc.n_tiles).astype(np.float32)
    sc.albedo = np.ascontiguousarray(rho_tile[sc.tile])       # per-tile albedo: beta uses the right surface
    L = scenes.make_lights([scenes.spot_light((0.45, 0.5, 0.92), 0.3, -1.35, 1.0, 0.45, 0.9)])
    Lt = scenes.perturb_lights(L, seed=7, pos_sigma=0.05)
    target = oracle.forward(sc, Lt, 101, 1 << 14, 3)["E"]
    alpha = np.random.default_rng(2).uniform(0.5, 1.5, sc.n_texels)
    return sc, L, target, alpha


@pytest.mark.parametrize("k,h", [(5, 1e-5), (6, 1e-6)])
def test_fd_exact_parameters_match_adjoint_spot(k, h):
    sc, L, target, alpha = _cornell_spot_setup()
    n, B, seed = 1 << 14, 3, 2
    O, w = _objective(sc, L, seed, n, B, target, alpha)
    g, segs = oracle.adjoint(sc, L, seed, n, B, w)
    Lp, Lm = L.copy(), L.copy()
    Lp[0, 1 + k] += h
    Lm[0, 1 + k] -= h
    fd = (_objective(sc, Lp, seed, n, B, target, alpha)[0] - _objective(sc, Lm, seed, n, B, target, alpha)[0]) / (2 * h)
    assert abs(g[0, k]) > 1e-8
    assert g[0, k] == pytest.approx(fd, rel=1e-6)


def test_fd_exact_intensity_matches_adjoint_point_cornell():
    sc = scenes.cornell_box(res=16)
    L = scenes.cornell_lights()
    Lt = scenes.perturb_lights(L, seed=1, pos_sigma=0.05)
    target = oracle.forward(sc, Lt, 101, 1 << 14, 3)["E"]
    alpha = np.ones(sc.n_texels)
    n, B, seed, h = 1 << 14, 3, 2, 1e-6
    O, w = _objective(sc, L, seed, n, B, target, alpha)
    g, _ = oracle.adjoint(sc, L, seed, n, B, w)
    Lp, Lm = L.copy(), L.copy()
    Lp[0, 6] += h
    Lm[0, 6] -= h
    fd = (_objective(sc, Lp, seed, n, B, target, alpha)[0] - _objective(sc, Lm, seed, n, B, target, alpha)[0]) / (2 * h)
    assert g[0, 5] == pytest.approx(fd, rel=1e-6)
    # a point light has no orientation or cone gradient
    assert np.all(g[0, 3:5] == 0) and np.all(g[0, 6:] == 0)


def _batched_adjoint(sc, L, seed, n, B, w, batches):
    per = n // batches
    parts = []
    for b in range(batches):
        g, _ = oracle.adjoint(sc, L, seed, n, B, w, begin=b * per, end=(b + 1) * per)
        parts.append(g[0] * batches)
    parts = np.array(parts)
    return parts.mean(0), parts.std(0, ddof=1) / np.sqrt(batches)


def _ramp_weights(res):
    u = (np.arange(res) + 0.5) / res
    U, V = np.meshgrid(u, u, indexing="xy")
    return (1.0 + 0.8 * (U - 0.5) + 0.6 * (V - 0.3) ** 2).reshape(-1)


def test_point_light_position_gradient_matches_closed_form():
    half, res, I = 1.0, 8, 1.5
    pos = np.array([0.2, -0.15, 0.7])
    sc = scenes.plane(half=half, res=res)
    L = scenes.make_lights([scenes.point_light(pos, I)])
    w = _ramp_weights(res)
    n = 1 << 22
    G, s = _batched_adjoint(sc, L, 3, n, 1, w, 16)

    def F(p):      # sum_t w_t A_t E_t = I sum_t w_t Omega_t
        return I * np.sum(w * cf.plane_texel_solid_angles(half, res, p))

    h = 1e-5
    for k in range(3):
        e = np.zeros(3); e[k] = h
        fd = (F(pos + e) - F(pos - e)) / (2 * h)
        assert abs(G[k] - fd) <= max(4.5 * s[k], 1e-3 * abs(fd)), (k, G[k], fd, s[k])
    p = np.sqrt(2 * I)
    assert G[5] == pytest.approx(p * np.sum(w * cf.plane_texel_solid_angles(half, res, pos)), rel=4.5 * s[5] / abs(G[5]) + 1e-3)


def test_spot_gradients_match_quadrature():
    half, res = 1.5, 8
    light = np.array(scenes.spot_light((0.1, 0.2, 1.0), 0.4, -np.pi / 2 + 0.5, 2.0, 0.25, 0.7))
    sc = scenes.plane(half=half, res=res)
    L = scenes.make_lights([light])
    w = _ramp_weights(res)
    n = 1 << 22
    G, s = _batched_adjoint(sc, L, 4, n, 1, w, 16)

    def F(row):
        return np.sum(w * cf.plane_texel_spot_flux(half, res, row, sub=8, order=6))

    steps = {0: 1e-4, 1: 1e-4, 2: 1e-4, 3: 1e-4, 4: 1e-4, 5: 1e-4, 6: 1e-4, 7: 1e-4}
    for k, h in steps.items():
        rp, rm = light.copy(), light.copy()
        rp[1 + k] += h
        rm[1 + k] -= h
        fd = (F(rp) - F(rm)) / (2 * h)
        assert abs(G[k] - fd) <= max(4.5 * s[k], 2e-3 * abs(fd)), (k, G[k], fd, s[k])
    # the position, orientation and cone gradients are all exercised
    assert np.all(np.abs(G) > 5 * s), (G, s)


def test_symmetric_light_has_no_lateral_gradient():
    half, res = 1.0, 8
    sc = scenes.plane(half=half, res=res)
    L = scenes.make_lights([scenes.point_light((0.0, 0.0, 0.8), 1.0)])
    n = 1 << 20
    E = oracle.forward(sc, L, 9, n, 1)["E"]
    O, w = oracle.loss(sc, E, np.zeros_like(E), np.ones_like(E))
    G, s = _batched_adjoint(sc, L, 9, n, 1, w, 16)
    assert abs(G[0]) < 4.5 * s[0] and abs(G[1]) < 4.5 * s[1]
    assert G[2] < -10 * s[2]


def test_loss_on_a_hand_computed_case():
    b = scenes._Builder()
    b.triangle([0, 0, 0], [2, 0, 0], [0, 2, 0], 0.5)        # area 2
    b.triangle([0, 0, 1], [3, 0, 1], [0, 2, 1], 0.5)        # area 3
    sc = b.build("two")
    O, w = oracle.loss(sc, [1.0, 2.0], [0.5, 3.0], [1.0, 0.5])
    assert O == pytest.approx(0.5 * (2 * 1 * 0.25 + 3 * 0.5 * 1.0))
    np.testing.assert_allclose(w, [0.5, -0.5])


def test_photon_ranges_partition_the_passes():
    sc = scenes.cornell_box(res=8)
    L = scenes.make_lights([scenes.point_light((0.5, 0.5, 0.9), 1.0),
                            scenes.spot_light((0.3, 0.3, 0.9), 0.1, -1.4, 2.0, 0.3, 0.6)])
    n, B = 10001, 3
    full = oracle.forward(sc, L, 5, n, B)
    cut = [0, 3000, 7777, n]
    parts = sum(oracle.forward(sc, L, 5, n, B, begin=a, end=b)["E"] for a, b in zip(cut[:-1], cut[1:]))
    np.testing.assert_allclose(parts, full["E"], rtol=1e-12, atol=1e-300)
    one = oracle.forward(sc, L, 5, n, B, threads=1)
    four = oracle.forward(sc, L, 5, n, B, threads=4)
    assert np.array_equal(one["E"], four["E"]) and np.array_equal(one["E"], full["E"])
    w = np.random.default_rng(0).normal(size=sc.n_texels)
    g_full, _ = oracle.adjoint(sc, L, 5, n, B, w)
    g_parts = sum(oracle.adjoint(sc, L, 5, n, B, w, begin=a, end=b)[0] for a, b in zip(cut[:-1], cut[1:]))
    np.testing.assert_allclose(g_parts, g_full, rtol=1e-10, atol=1e-14)
    g1, _ = oracle.adjoint(sc, L, 5, n, B, w, threads=1)
    g3, _ = oracle.adjoint(sc, L, 5, n, B, w, threads=3)
    assert np.array_equal(g1, g3)
