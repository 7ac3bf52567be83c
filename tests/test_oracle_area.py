"""Pins of the oracle's rectangular area lights (supplement, Eq. S.15-S.16):
sampling distributions, the flux normalisation (expected total = the power
P), exact energy bookkeeping in a closed box, the one-bounce irradiance on a
plane against 4-D Gauss-Legendre quadrature of the Lambertian emitter, the
flux derivative against central differences of its definition, the adjoint
against finite differences of the quadrature objective, and the same-seed
finite difference of the power through several bounces."""
import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2310_02043_gb300 import scenes
from tests import closed_forms as cf


def _frame(yaw, pitch):
    n = cf.spot_axis(yaw, pitch)
    t = np.array([-np.sin(pitch) * np.cos(yaw), -np.sin(pitch) * np.sin(yaw), np.cos(pitch)])
    return n, t, np.cross(n, t)


def test_emission_samples_the_rectangle_and_the_hemisphere():
    row = np.array(scenes.area_light((0.3, -0.2, 1.0), 0.7, -1.2, 3.0, 0.6, 0.4))
    n_rays = 20000
    n, t, b = _frame(0.7, -1.2)
    W, X0, PHI, A = [], [], [], []
    for k in range(n_rays):
        w, phi, a, x0 = oracle.emit(row, n_rays, 11, k, origin=True)
        W.append(w); X0.append(x0); PHI.append(phi); A.append(a)
    W, X0, PHI, A = map(np.array, (W, X0, PHI, A))
    d = X0 - row[1:4]
    assert np.abs(d @ n).max() < 1e-12                        # origins lie in the light's plane
    su, sv = d @ t, d @ b
    assert stats.kstest((su + 0.3) / 0.6, "uniform").pvalue > 1e-3
    assert stats.kstest((sv + 0.2) / 0.4, "uniform").pvalue > 1e-3
    c = W @ n
    assert np.all(c > 0) and np.allclose(np.linalg.norm(W, axis=1), 1.0)
    assert stats.kstest(c, "uniform").pvalue > 1e-3           # uniform hemisphere: cos uniform
    az = np.arctan2(W @ b, W @ t)
    assert stats.kstest((az + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-3
    assert np.allclose(A, c, rtol=1e-12)
    P = 3.0
    assert np.allclose(PHI, 2 * P * c / n_rays, rtol=1e-12)
    assert abs(PHI.sum() - P) < 5 * 2 * P * np.sqrt(1 / 12) / np.sqrt(n_rays)


def test_closed_box_receives_every_emitted_ray():
    sc = scenes.closed_cube(res=4, albedo=0.6)
    row = np.array(scenes.area_light((0.5, 0.45, 0.55), 0.3, 0.4, 2.0, 0.3, 0.2))
    n = 4096
    f1 = oracle.forward(sc, row[None], 3, n, 1)
    A = oracle.texel_areas(sc)
    emitted = sum(oracle.emit(row, n, 3, k)[1] for k in range(n))
    assert np.sum(A * f1["E"]) == pytest.approx(emitted, rel=1e-12)
    f2 = oracle.forward(sc, row[None], 3, n, 2)
    assert np.sum(A * f2["E"]) == pytest.approx(emitted * (1 + float(np.float32(0.6))), rel=1e-12)


def _plane_flux_quadrature(half, res, row, sub=4, order=3, lsub=4, lorder=4):
    """Int_texel Int_light P/(pi A) cos_e cos_r / r^2 dA dA' for every texel of
    the plane z = 0 (the texel's one-bounce flux), Gauss-Legendre in 4-D."""
    _, x, y, z, yaw, pitch, p, wd, ht = row
    P = 0.5 * p * p
    n, t, b = _frame(yaw, pitch)
    g, gw = np.polynomial.legendre.leggauss(lorder)
    lc = -0.5 + (np.arange(lsub) + 0.5) / lsub
    lu = (lc[:, None] + 0.5 / lsub * g[None, :]).ravel()
    lw = np.tile(0.5 / lsub * gw, lsub)
    U, V = np.meshgrid(lu * wd, lu * ht, indexing="xy")
    WU, WV = np.meshgrid(lw * wd, lw * ht, indexing="xy")
    Lp = np.array([x, y, z])[None, :] + U.reshape(-1, 1) * t + V.reshape(-1, 1) * b
    Lw = (WU * WV).reshape(-1)
    g2, gw2 = np.polynomial.legendre.leggauss(order)
    cells = res * sub
    h = 2 * half / cells
    centers = -half + (np.arange(cells) + 0.5) * h
    nodes = (centers[:, None] + 0.5 * h * g2[None, :]).reshape(-1)
    weights = np.tile(0.5 * h * gw2, cells)
    X, Y = np.meshgrid(nodes, nodes, indexing="xy")
    WX, WY = np.meshgrid(weights, weights, indexing="xy")
    R = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], 1)
    d = R[:, None, :] - Lp[None, :, :]
    r2 = np.sum(d * d, axis=2)
    r = np.sqrt(r2)
    ce = np.maximum(np.einsum("ijk,k->ij", d, n) / r, 0.0)
    cr = np.abs(d[:, :, 2]) / r
    f = (P / (np.pi * wd * ht)) * ce * cr / r2 @ Lw
    f = (f * (WX * WY).ravel()).reshape(X.shape)
    m = cells * order
    return f.reshape(res, m // res, res, m // res).sum(axis=(1, 3)).reshape(-1)


def test_one_bounce_irradiance_matches_quadrature():
    half, res = 1.5, 8
    row = np.array(scenes.area_light((0.1, 0.2, 1.0), 0.4, -np.pi / 2 + 0.3, 2.0, 0.5, 0.3))
    sc = scenes.plane(half=half, res=res)
    f = oracle.forward(sc, row[None], 5, 1 << 21, 1, counts=True)
    A = oracle.texel_areas(sc)
    ref = _plane_flux_quadrature(half, res, row) / A
    sigma = f["E"] / np.sqrt(np.maximum(f["count"], 1))
    lit = ref > 0.05 * ref.max()
    assert np.all(np.abs(f["E"] - ref)[lit] < 5 * sigma[lit] + 2e-3 * ref[lit])
    assert np.sum(A * f["E"]) == pytest.approx(np.sum(A * ref), rel=5e-3)


def test_flux_derivative_matches_its_definition():
    # dPhi_r/dq = Phi_r d log(cos_theta cos_1 / r^2)/dq with x1 fixed and the
    # origin at fixed local coordinates: central differences of that product
    row = np.array(scenes.area_light((0.2, -0.1, 1.1), 0.5, -1.3, 1.7, 0.6, 0.35))
    x1 = np.array([0.4, 0.3, 0.0])
    n1 = np.array([0.0, 0.0, 1.0])
    u3, u4, N = 0.8, 0.25, 1000

    def h(r):
        n, t, b = _frame(r[4], r[5])
        x0 = r[1:4] + (2 * u3 - 1) * 0.5 * r[7] * t + (2 * u4 - 1) * 0.5 * r[8] * b
        d = x1 - x0
        dist = np.linalg.norm(d)
        w = d / dist
        return 0.5 * r[6] ** 2 * 2 * (n @ w) / N * (n1 @ -w) / dist ** 2

    phi, g = oracle.dflux(row, N, x1, n1, u3=u3, u4=u4)
    n, t, b = _frame(row[4], row[5])
    x0 = row[1:4] + (2 * u3 - 1) * 0.3 * t + (2 * u4 - 1) * 0.175 * b
    d = x1 - x0
    scale = np.linalg.norm(d) ** 2 / (n1 @ -(d / np.linalg.norm(d)))
    assert phi == pytest.approx(2 * 1.7 * (n @ d) / np.linalg.norm(d) / N, rel=1e-12)    # 2 P cos / N
    for k, col in enumerate([1, 2, 3, 4, 5, 6]):
        e = 1e-6
        rp, rm = row.copy(), row.copy()
        rp[col] += e
        rm[col] -= e
        fd = scale * (h(rp) - h(rm)) / (2 * e)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-12), (col, g[k], fd)
    assert g[6] == 0 and g[7] == 0


def _ramp_weights(res):
    u = (np.arange(res) + 0.5) / res
    U, V = np.meshgrid(u, u, indexing="xy")
    return (1.0 + 0.8 * (U - 0.5) + 0.6 * (V - 0.3) ** 2).reshape(-1)


def test_area_gradients_match_quadrature():
    half, res = 1.5, 8
    row = np.array(scenes.area_light((0.1, 0.2, 1.0), 0.4, -np.pi / 2 + 0.3, 2.0, 0.5, 0.3))
    sc = scenes.plane(half=half, res=res)
    w = _ramp_weights(res)
    n, batches = 1 << 22, 16
    per = n // batches
    parts = np.array([oracle.adjoint(sc, row[None], 4, n, 1, w, begin=k * per, end=(k + 1) * per)[0][0] * batches
                      for k in range(batches)])
    G, s = parts.mean(0), parts.std(0, ddof=1) / np.sqrt(batches)

    def F(r):
        return np.sum(w * _plane_flux_quadrature(half, res, r))

    for k in range(6):
        rp, rm = row.copy(), row.copy()
        e = 1e-4
        rp[1 + k] += e
        rm[1 + k] -= e
        fd = (F(rp) - F(rm)) / (2 * e)
        assert abs(G[k] - fd) <= max(4.5 * s[k], 3e-3 * abs(fd)), (k, G[k], fd, s[k])
    assert np.all(G[6:] == 0)
    assert np.all(np.abs(G[:6]) > 5 * s[:6]), (G, s)


def test_power_gradient_is_the_same_seed_finite_difference():
    sc = scenes.cornell_box(res=8)
    row = np.array(scenes.area_light((0.5, 0.5, 0.95), 0.3, -np.pi / 2 + 0.1, 1.5, 0.2, 0.15))
    L = row[None]
    rng = np.random.default_rng(3)
    target = rng.uniform(0, 1, sc.n_texels)
    alpha = np.ones(sc.n_texels)
    n, B = 1 << 14, 3
    E = oracle.forward(sc, L, 7, n, B)["E"]
    _, w = oracle.loss(sc, E, target, alpha)
    g, _ = oracle.adjoint(sc, L, 7, n, B, w)
    h = 1e-5
    Lp, Lm = L.copy(), L.copy()
    Lp[0, 6] += h
    Lm[0, 6] -= h
    Op = oracle.loss(sc, oracle.forward(sc, Lp, 7, n, B)["E"], target, alpha)[0]
    Om = oracle.loss(sc, oracle.forward(sc, Lm, 7, n, B)["E"], target, alpha)[0]
    assert g[0, 5] == pytest.approx((Op - Om) / (2 * h), rel=1e-6)
