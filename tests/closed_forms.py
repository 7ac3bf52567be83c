"""Closed-form and quadrature references used to pin the oracle.

These are textbook results written independently of the oracle:
solid angle of a rectangle seen from a point above its plane, solid angle of
a triangle (Van Oosterom and Strackee, 1983), and Gauss-Legendre quadrature
of the spot's irradiance a(theta) cos / r^2 over a texel."""
import numpy as np


def rect_solid_angle(x0, x1, y0, y1, p):
    """Solid angle of the rectangle [x0,x1]x[y0,y1] in the plane z = 0 seen
    from p = (px, py, h), h > 0: signed corner sum of
    atan(a b / (h sqrt(a^2 + b^2 + h^2)))."""
    px, py, h = p

    def F(a, b):
        return np.arctan(a * b / (h * np.sqrt(a * a + b * b + h * h)))

    a0, a1, b0, b1 = x0 - px, x1 - px, y0 - py, y1 - py
    return F(a1, b1) - F(a0, b1) - F(a1, b0) + F(a0, b0)


def plane_texel_solid_angles(half, res, p):
    """Solid angle of every texel of the square plane [-half, half]^2 (texel
    index iu + res iv)."""
    edges = np.linspace(-half, half, res + 1)
    x0, x1 = edges[:-1][None, :], edges[1:][None, :]
    y0, y1 = edges[:-1][:, None], edges[1:][:, None]
    return rect_solid_angle(x0, x1, y0, y1, p).reshape(-1)


def triangle_solid_angle(a, b, c, p):
    """Van Oosterom-Strackee: tan(Omega/2) = |R1.(R2xR3)| /
    (r1 r2 r3 + (R1.R2) r3 + (R1.R3) r2 + (R2.R3) r1)."""
    R1, R2, R3 = np.asarray(a) - p, np.asarray(b) - p, np.asarray(c) - p
    r1, r2, r3 = np.linalg.norm(R1), np.linalg.norm(R2), np.linalg.norm(R3)
    num = abs(np.dot(R1, np.cross(R2, R3)))
    den = r1 * r2 * r3 + np.dot(R1, R2) * r3 + np.dot(R1, R3) * r2 + np.dot(R2, R3) * r1
    return 2.0 * np.arctan2(num, den)


def spot_axis(yaw, pitch):
    return np.array([np.cos(pitch) * np.cos(yaw), np.cos(pitch) * np.sin(yaw), np.sin(pitch)])


def spot_quadratic_falloff(c, ci, co):
    """Supplement Eq. S.11, quadratic in cos(theta) between the cones."""
    s = np.clip((c - co) / (ci - co), 0.0, 1.0)
    return s * s


def plane_texel_spot_flux(half, res, light, sub=8, order=4):
    """Int_texel I a(theta) cos / r^2 dA for every texel of the plane z = 0
    (the light's irradiance times the texel area), by Gauss-Legendre quadrature
    on sub x sub cells per texel with order x order nodes each."""
    _, x, y, z, yaw, pitch, p, th_in, th_out = light
    I = 0.5 * p * p
    n = spot_axis(yaw, pitch)
    ci, co = np.cos(th_in), np.cos(th_out)
    g, gw = np.polynomial.legendre.leggauss(order)
    cells = res * sub
    h = 2 * half / cells
    centers = -half + (np.arange(cells) + 0.5) * h
    nodes = (centers[:, None] + 0.5 * h * g[None, :]).reshape(-1)
    weights = np.tile(0.5 * h * gw, cells)
    X, Y = np.meshgrid(nodes, nodes, indexing="xy")
    WX, WY = np.meshgrid(weights, weights, indexing="xy")
    dx, dy, dz = X - x, Y - y, 0.0 - z
    r2 = dx * dx + dy * dy + dz * dz
    r = np.sqrt(r2)
    c = (n[0] * dx + n[1] * dy + n[2] * dz) / r
    cos_recv = np.abs(dz) / r
    f = I * spot_quadratic_falloff(c, ci, co) * cos_recv / r2 * WX * WY
    m = res * sub * order
    per = f.reshape(res, m // res, res, m // res).sum(axis=(1, 3))
    return per.reshape(-1)
