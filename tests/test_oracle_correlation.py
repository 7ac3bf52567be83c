"""Correlated and decorrelated adjoint estimates (Sec. 4.3), pinned by their
exact expectations.

A point light over a plane, one hit, N photons, the objective
O = 1/2 sum_t A_t (E_t - E*_t)^2 with E* half the light's own irradiance.
The adjoint weights w_t = E^_t - E*_t come from a forward estimate E^.

* Decorrelated (the adjoint replays other photons than the forward pass):
  w and the replayed paths are independent, so the estimate is unbiased:
  its mean is dO/dp.
* Correlated (the same photons): the texel flux F^_t = A_t E^_t and the
  estimate D^_t of dF_t/dp are sums over the same i.i.d. photons, and a
  photon carrying phi = 4 pi I / N into texel t contributes to both, so
  Cov(F^_t, D^_t) = phi (1 - p_t) dF_t/dp with p_t = Omega_t / (4 pi). The
  mean is then dO/dp + (4 pi I / N) sum_t (1 - p_t) / A_t * I dOmega_t/dp,
  a bias that falls as 1/N.

Both expectations come from the closed-form solid angles of the texels;
the sample means of thousands of estimates must match them."""
import numpy as np

import oracle
from paper_2310_02043_gb300 import scenes
from tests import closed_forms as cf

HALF, RES, I = 1.0, 4, 1.0
POS = np.array([0.3, -0.2, 0.5])
H = 1e-5


def _omega(p):
    return cf.plane_texel_solid_angles(HALF, RES, p)


def _d_omega(p):
    return np.array([(_omega(p + H * e) - _omega(p - H * e)) / (2 * H) for e in np.eye(3)])    # [3, texels]


def test_decorrelated_is_unbiased_and_correlated_bias_is_the_covariance():
    sc = scenes.plane(half=HALF, res=RES)
    A = oracle.texel_areas(sc)
    E = I * _omega(POS) / A
    E_star = 0.5 * E
    dE = I * _d_omega(POS) / A
    g_true = np.sum(A * (E - E_star) * dE, axis=1)                 # dO/dp for x, y, z
    L = scenes.make_lights([scenes.point_light(POS, I)])
    K = 4000
    for n in (1 << 8, 1 << 10):
        p = _omega(POS) / (4 * np.pi)
        bias = (4 * np.pi * I / n) * np.sum((1 - p) / A * I * _d_omega(POS), axis=1)
        corr, decorr = [], []
        for k in range(K):
            w = oracle.forward(sc, L, 1000 + k, n, 1)["E"] - E_star
            corr.append(oracle.adjoint(sc, L, 1000 + k, n, 1, w)[0][0, :3])
            decorr.append(oracle.adjoint(sc, L, 500000 + k, n, 1, w)[0][0, :3])
        for g, expect in ((np.array(corr), g_true + bias), (np.array(decorr), g_true)):
            m, s = g.mean(0), g.std(0, ddof=1) / np.sqrt(K)
            assert np.all(np.abs(m - expect) <= 4.5 * s), (n, m, expect, s)
        # the covariance term is resolved: at 256 photons it is many sigma along z
        s_corr = np.array(corr).std(0, ddof=1) / np.sqrt(K)
        if n == 1 << 8:
            assert abs(bias[2]) > 8 * s_corr[2], (bias, s_corr)
