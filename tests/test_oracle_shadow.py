"""The estimator's known limit at moving shadows, pinned by quadrature.

The adjoint (Alg. 2 with Eq. 11 and 14) differentiates each photon's flux
with its first hit x1 held fixed, so visibility is held fixed: what it
estimates is the derivative of the objective with the shadow frozen where it
was. A point light above a floor partly shadowed by a square occluder, one
hit, the objective 1/2 sum_floor A_t E_t^2 (adjoint weights from quadrature
irradiance): the oracle's adjoint must match central differences of the
frozen-visibility quadrature objective on every axis, and it must differ
from the derivative with visibility recomputed, whose shadow outline moves
with the light on every axis (the boundary term the method leaves out)."""
import numpy as np

import oracle
from paper_2310_02043_gb300 import scenes

HALF, RES, ZO, OC, OH = 1.5, 8, 0.4, (0.1, 0.0), 0.25


def _rect_flux(light, x0, x1, y0, y1, intensity, order=8, sub=2):
    """Integral of I cos / r^2 = I z_l / r^3 over the floor rectangles
    [x0, x1] x [y0, y1] (arrays; empty where x1 <= x0 or y1 <= y0), by a
    Gauss-Legendre product rule on sub x sub cells of each rectangle."""
    g, gw = np.polynomial.legendre.leggauss(order)
    t = ((np.arange(sub)[:, None] + 0.5 + 0.5 * g[None, :]) / sub).ravel()
    wt = np.tile(gw, sub) * 0.5 / sub
    wx, wy = np.maximum(x1 - x0, 0.0), np.maximum(y1 - y0, 0.0)
    X = x0[:, None] + wx[:, None] * t[None, :]
    Y = y0[:, None] + wy[:, None] * t[None, :]
    dx, dy = light[0] - X[:, :, None], light[1] - Y[:, None, :]
    f = intensity * light[2] / (dx * dx + dy * dy + light[2] ** 2) ** 1.5
    return np.einsum("tij,i,j->t", f, wt, wt) * wx * wy


def _floor_irradiance(light, vis_light, intensity=1.0):
    """Texel-average irradiance of the floor from a point light at `light`,
    shadowed by the occluder as seen from `vis_light`. The shadow of the
    horizontal square on the floor is the axis-aligned square it projects
    to, so each texel's flux is the integral over the texel minus the
    integral over its overlap with the shadow: two smooth integrands, no
    quadrature across the outline."""
    light, vis_light = np.asarray(light, np.float64), np.asarray(vis_light, np.float64)
    edges = np.linspace(-HALF, HALF, RES + 1)
    x0, y0 = np.meshgrid(edges[:-1], edges[:-1], indexing="xy")
    x1, y1 = np.meshgrid(edges[1:], edges[1:], indexing="xy")
    x0, y0, x1, y1 = x0.ravel(), y0.ravel(), x1.ravel(), y1.ravel()     # texel ix + RES iy
    s = vis_light[2] / (vis_light[2] - ZO)                                # projection onto z = 0
    sx = vis_light[0] + (np.array([OC[0] - OH, OC[0] + OH]) - vis_light[0]) * s
    sy = vis_light[1] + (np.array([OC[1] - OH, OC[1] + OH]) - vis_light[1]) * s
    lit = _rect_flux(light, x0, x1, y0, y1, intensity)
    dark = _rect_flux(light, np.maximum(x0, sx[0]), np.minimum(x1, sx[1]), np.maximum(y0, sy[0]),
                      np.minimum(y1, sy[1]), intensity)
    return (lit - dark) / (2 * HALF / RES) ** 2


def test_adjoint_is_the_frozen_visibility_derivative():
    sc = scenes.occluded_plane(HALF, RES, ZO, OC, OH)
    L = scenes.make_lights([scenes.point_light((0.2, 0.1, 1.0), 1.0)])
    x0 = L[0, 1:4].copy()
    A = oracle.texel_areas(sc)
    nf = RES * RES
    E0 = _floor_irradiance(x0, x0)
    w = np.zeros(sc.n_texels)
    w[:nf] = E0                                    # alpha = 1 on the floor, 0 on the occluder; target 0

    def objective(x, frozen):
        E = _floor_irradiance(x, x0 if frozen else x)
        return 0.5 * np.sum(A[:nf] * E * E)

    def central(axis, h, frozen):
        xp, xm = x0.copy(), x0.copy()
        xp[axis] += h
        xm[axis] -= h
        return (objective(xp, frozen) - objective(xm, frozen)) / (2 * h)

    n, batches = 1 << 22, 16
    per = n // batches
    parts = np.array([oracle.adjoint(sc, L, 3, n, 1, w, begin=k * per, end=(k + 1) * per)[0][0] * batches
                      for k in range(batches)])
    G, sigma = parts.mean(0), parts.std(0, ddof=1) / np.sqrt(batches)
    for axis in range(3):
        frozen = central(axis, 1e-2, True)
        assert abs(frozen - central(axis, 1e-3, True)) <= 1e-3 * abs(frozen)     # smooth: a plateau in h
        assert abs(G[axis] - frozen) <= 4.0 * sigma[axis] + 2e-3 * abs(frozen), (axis, G[axis], frozen, sigma[axis])
        # the shadow outline moves with the light: the full derivative
        # carries a boundary term that the frozen one, and the adjoint, leave out
        full = central(axis, 1e-2, False)
        assert abs(full - central(axis, 1e-3, False)) <= 1e-3 * abs(full)
        assert abs(full - G[axis]) > 20.0 * sigma[axis], (axis, full, G[axis], sigma[axis])
        assert abs(full - frozen) > 0.3 * abs(full)


def test_forward_irradiance_in_the_shadow_matches_quadrature():
    """The traced floor irradiance (Alg. 1, Eq. 8) with the occluder's
    shadow: hard outline, umbra with E = 0, against the quadrature."""
    sc = scenes.occluded_plane(HALF, RES, ZO, OC, OH)
    L = scenes.make_lights([scenes.point_light((0.2, 0.1, 1.0), 1.0)])
    E = oracle.forward(sc, L, 5, 1 << 22, 1)["E"][:RES * RES]
    Q = _floor_irradiance(L[0, 1:4], L[0, 1:4])
    assert Q.min() < 0.5 * Q.max()                 # the shadow is on the floor
    assert np.max(np.abs(E - Q)) <= 0.03 * Q.max()
