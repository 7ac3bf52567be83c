"""The estimator's known limit at moving shadows, pinned by quadrature.

The adjoint (Alg. 2 with Eq. 11 and 14) differentiates each photon's flux
with its first hit x1 held fixed, so visibility is held fixed: what it
estimates is the derivative of the objective with the shadow frozen where it
was. A point light above a floor partly shadowed by a square occluder, one
hit, the objective 1/2 sum_floor A_t E_t^2 (adjoint weights from quadrature
irradiance): the oracle's adjoint must match central differences of the
frozen-visibility quadrature objective on every axis, and it must differ
from the derivative with visibility recomputed along z, where the shadow
outline moves with the light (the boundary term the method leaves out)."""
import numpy as np

import oracle
from paper_2310_02043_gb300 import scenes

HALF, RES, ZO, OC, OH = 1.5, 8, 0.4, (0.1, 0.0), 0.25


def _floor_irradiance(light, vis_light, intensity=1.0, sub=16, order=4):
    """Texel-average irradiance I cos / r^2 of the floor by Gauss-Legendre
    quadrature, a point shadowed when the segment to vis_light crosses the
    occluder square."""
    g, gw = np.polynomial.legendre.leggauss(order)
    cells = RES * sub
    h = 2 * HALF / cells
    c = -HALF + (np.arange(cells) + 0.5) * h
    nodes = (c[:, None] + 0.5 * h * g[None, :]).ravel()
    wts = np.tile(0.5 * h * gw, cells)
    X, Y = np.meshgrid(nodes, nodes, indexing="xy")
    WX, WY = np.meshgrid(wts, wts, indexing="xy")
    dx, dy, dz = light[0] - X, light[1] - Y, np.full_like(X, light[2])
    r2 = dx * dx + dy * dy + dz * dz
    cos = dz / np.sqrt(r2)
    s = ZO / vis_light[2]
    qx, qy = X + s * (vis_light[0] - X), Y + s * (vis_light[1] - Y)
    visible = ~((np.abs(qx - OC[0]) < OH) & (np.abs(qy - OC[1]) < OH))
    f = intensity * cos / r2 * visible * WX * WY
    m = cells * order
    return f.reshape(RES, m // RES, RES, m // RES).sum(axis=(1, 3)).reshape(-1) / (2 * HALF / RES) ** 2


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
    # along z the shadow outline moves with the light: the full derivative
    # carries a boundary term that the frozen one, and the adjoint, leave out
    full_z = central(2, 1e-2, False)
    assert abs(full_z - G[2]) > 50.0 * sigma[2], (full_z, G[2], sigma[2])
    assert abs(full_z - central(2, 1e-2, True)) > 0.1 * abs(full_z)


def test_forward_irradiance_in_the_shadow_matches_quadrature():
    """The traced floor irradiance (Alg. 1, Eq. 8) with the occluder's
    shadow: hard outline, umbra with E = 0, all of it from quadrature."""
    sc = scenes.occluded_plane(HALF, RES, ZO, OC, OH)
    L = scenes.make_lights([scenes.point_light((0.2, 0.1, 1.0), 1.0)])
    E = oracle.forward(sc, L, 5, 1 << 22, 1)["E"][:RES * RES]
    Q = _floor_irradiance(L[0, 1:4], L[0, 1:4])
    assert Q.min() < 0.5 * Q.max()                 # the shadow is on the floor
    assert np.max(np.abs(E - Q)) <= 0.03 * Q.max()
