"""Pins of the surrogate oracle (oracle/surrogate.py) against what the
mathematics and independent library routines fix: bf16 rounding against
torch's conversion, the hash encoding's exact reproduction of linear fields
and its adjoint identity, the published hash at hand-computed vertices, every
derivative against float64 central differences, the network against torch's
autograd, Adam against torch.optim.Adam, the direct term against the traced
irradiance of a spot over a plane, texel centres against the analytic grid."""
import numpy as np
import pytest
import torch

import oracle
from oracle import surrogate as S
from paper_2310_02043_gb300 import scenes

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _rng(seed=0):
    return np.random.default_rng(seed)


def test_bf16_matches_torch_and_ties_to_even():
    x = _rng().normal(size=5000) * np.exp(_rng(1).uniform(-20, 20, 5000))
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(S.bf16(x), ref)
    assert S.bf16(1.0 + 2.0 ** -8) == 1.0                   # halfway, even neighbour is 1
    assert S.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6    # halfway, even neighbour above
    assert S.bf16(1.0 + 0.75 * 2.0 ** -7) == 1.0 + 2.0 ** -7


def test_levels_dense_then_hashed():
    assert [S.dense_level(l) for l in range(16)] == [True] * 7 + [False] * 9
    assert S.RES[0] == 16 and S.RES[-1] == 512
    for l, n in enumerate(S.RES):
        assert n == int(np.floor(16 * 2.0 ** (l / 3) + 1e-9))


def test_hash_at_hand_computed_vertices():
    # (x * 1) xor (y * 2654435761) xor (z * 805459861), low 19 bits
    v = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [3, 5, 7], [511, 1, 300]])
    got = S.vertex_index(15, v)
    assert got.tolist() == [1, 0x9E3779B1 & 0x7FFFF, 0x30025795 & 0x7FFFF,
                            (3 ^ ((5 * 0x9E3779B1) & 0xFFFFFFFF) ^ ((7 * 0x30025795) & 0xFFFFFFFF)) & 0x7FFFF,
                            (511 ^ 0x9E3779B1 ^ ((300 * 0x30025795) & 0xFFFFFFFF)) & 0x7FFFF]
    # dense levels are a bijection of the grid onto the first (N+1)^3 slots
    n = S.RES[6] + 1
    g = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    idx = S.vertex_index(6, g)
    assert np.array_equal(np.sort(idx), np.arange(n ** 3))


def test_hash_spreads_a_level_over_the_table():
    l = 12
    g = _rng(2).integers(0, S.RES[l] + 1, size=(200000, 3))
    idx = S.vertex_index(l, g)
    counts = np.bincount(idx // (S.TABLE // 64), minlength=64)
    chi2 = np.sum((counts - counts.mean()) ** 2 / counts.mean())
    assert chi2 < 120                                        # 63 dof


def test_encoding_reproduces_linear_fields_on_dense_levels():
    rng = _rng(3)
    table = rng.normal(size=(16, S.TABLE, 2))
    coef = rng.normal(size=(16, 2, 3))
    for l in range(7):
        n = S.RES[l] + 1
        g = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
        idx = S.vertex_index(l, g)
        for j in range(2):
            table[l, idx, j] = g @ coef[l, j] + 0.25
    xn = rng.uniform(0, 1, size=(500, 3)).astype(np.float32)
    enc = S.encode(xn, table)
    for l in range(7):
        pos = (xn * np.float32(S.RES[l])).astype(np.float32).astype(np.float64)
        for j in range(2):
            assert np.allclose(enc[:, 2 * l + j], pos @ coef[l, j] + 0.25, rtol=0, atol=1e-9)


def test_encoding_at_vertices_reads_the_slot_and_is_continuous():
    rng = _rng(4)
    table = rng.normal(size=(16, S.TABLE, 2))
    l = 13
    v = rng.integers(1, S.RES[l] - 1, size=(50, 3))
    xn = (v / S.RES[l]).astype(np.float32)
    ok = np.all((xn * np.float32(S.RES[l])).astype(np.float32) == v.astype(np.float32), axis=1)
    enc = S.encode(xn[ok], table)
    assert np.allclose(enc[:, 2 * l:2 * l + 2], table[l, S.vertex_index(l, v[ok])])
    # across a cell face the two sides agree to first order
    x0 = np.array([[0.3, 0.2, 0.1]], np.float32)
    h = np.float32(1e-6)
    e_lo = S.encode(x0 - h, table)
    e_hi = S.encode(x0 + h, table)
    assert np.max(np.abs(e_hi - e_lo)) < 1e-2


def test_encoding_adjoint_identity():
    rng = _rng(5)
    table = rng.normal(size=(16, S.TABLE, 2))
    xn = rng.uniform(0, 1, size=(300, 3)).astype(np.float32)
    g = rng.normal(size=(300, 32))
    lhs = np.sum(g * S.encode(xn, table))
    rhs = np.sum(S.encode_backward(xn, g) * table)
    assert lhs == pytest.approx(rhs, rel=1e-12)


def _spot(x=3.0, y=2.0, z=2.6, yaw=0.7, pitch=-1.2, I=1.0, ti=0.5, to=1.0):
    return np.array(scenes.spot_light((x, y, z), yaw, pitch, I, ti, to), np.float64)


def _texels(n, seed=6):
    rng = _rng(seed)
    x = np.column_stack([rng.uniform(0, 6, n), rng.uniform(0, 4, n), rng.uniform(0, 1.0, n)])
    nt = rng.normal(size=(n, 3))
    nt /= np.linalg.norm(nt, axis=1, keepdims=True)
    return x, nt


def test_geometry_derivatives_against_central_differences():
    x, nt = _texels(400)
    light = _spot()
    lo, ext = np.array([-1.0, -1.0, -0.5]), 8.0
    G, dG, D, dD = S.geometry(light, x, nt, lo, ext)
    cols = [1, 2, 3, 4, 5, 7]
    for k, c in enumerate(cols):
        h = 1e-6
        lp, lm = light.copy(), light.copy()
        lp[c] += h
        lm[c] -= h
        Gp, _, Dp, _ = S.geometry(lp, x, nt, lo, ext)
        Gm, _, Dm, _ = S.geometry(lm, x, nt, lo, ext)
        # skip points whose falloff or |cos_r| kinks lie within the step
        a, ci, co = G[:, S.F_A - 32], np.cos(light[7]), np.cos(light[8])
        cosl = G[:, S.F_COSL - 32]
        smooth = (np.abs(cosl - ci) > 1e-4) & (np.abs(cosl - co) > 1e-4) & (G[:, S.F_COSR - 32] > 1e-4)
        fdG = (Gp - Gm) / (2 * h)
        fdD = (Dp - Dm) / (2 * h)
        assert np.allclose(dG[smooth, :, k], fdG[smooth], rtol=1e-5, atol=1e-6), c
        assert np.allclose(dD[smooth, k], fdD[smooth], rtol=1e-5, atol=1e-6 * np.abs(D).max()), c
        assert a.max() > 0


def test_geometry_values():
    light = _spot(x=1.0, y=1.0, z=2.0, yaw=0.0, pitch=-np.pi / 2, ti=0.3, to=0.6)
    x = np.array([[1.0, 1.0, 0.0], [1.5, 1.0, 0.0], [4.0, 1.0, 0.0]])
    nt = np.array([[0.0, 0.0, 1.0]] * 3)
    G, _, D, _ = S.geometry(light, x, nt, [0, 0, 0], 10.0)
    # straight below: a = 1, cos_r = 1, D = 1 / r^2 = 1/4
    assert D[0] == pytest.approx(0.25, rel=1e-12)
    assert np.allclose(G[0, 0:3], [0, 0, 1]) and G[0, S.F_R - 32] == pytest.approx(0.2)
    # 0.5 m off axis: cos = 2 / sqrt(4.25); theta = 14.0 deg < 0.3 rad inner cone
    r2 = 4.25
    assert D[1] == pytest.approx((2 / np.sqrt(r2)) / r2, rel=1e-12)
    # beyond the outer cone: nothing
    assert D[2] == 0.0 and G[2, S.F_A - 32] == 0.0


def test_direct_term_is_the_traced_one_bounce_irradiance():
    # a spot over a plane, one hit: the traced texel irradiance is I times the
    # texel average of D (8 x 8 midpoint quadrature per texel)
    sc = scenes.plane(half=1.0, res=16, albedo=0.5)
    light = np.array([_spot(x=0.0, y=0.0, z=1.0, yaw=0.3, pitch=-1.3, I=2.0, ti=0.35, to=0.7)])
    f = oracle.forward(sc, light, 9, 1 << 21, 1, counts=True)
    pos, nrm = S.texel_centres(sc)
    h = 2.0 / 16
    sub = (np.arange(8) + 0.5) / 8 * h - h / 2
    Dbar = np.zeros(sc.n_texels)
    for dx in sub:
        for dy in sub:
            Dbar += S.geometry(light[0], pos + [dx, dy, 0.0], nrm, pos.min(0), 2.0)[2] / 64
    I = 2.0
    sigma = f["E"] / np.sqrt(np.maximum(f["count"], 1))
    inner = Dbar > 0.3 * Dbar.max()
    err = np.abs(f["E"] - I * Dbar)[inner]
    assert np.all(err < 5 * sigma[inner] + 2e-3 * I * Dbar[inner])
    A = oracle.texel_areas(sc)
    assert abs(np.sum(A * f["E"]) - np.sum(A * I * Dbar)) < 2e-3 * np.sum(A * I * Dbar)


def _weights(seed=7, scale=0.25):
    rng = _rng(seed)
    return [S.bf16(rng.normal(size=s) * scale) for s in S.WEIGHT_SHAPES]


def test_network_matches_torch_autograd():
    rng = _rng(8)
    W = _weights()
    X = rng.normal(size=(64, 64))
    do = rng.normal(size=(64, 16))
    o, cache = S.mlp_forward(X, W, rounding=False)
    dX, dW = S.mlp_backward(cache, W, do, rounding=False)
    Xt = torch.tensor(X, requires_grad=True)
    Wt = [torch.tensor(w, requires_grad=True) for w in W]
    h = Xt
    for k in range(3):
        h = torch.relu(h @ Wt[k].T)
    ot = h @ Wt[3].T
    (ot * torch.tensor(do)).sum().backward()
    assert np.allclose(o, ot.detach().numpy(), rtol=1e-12, atol=1e-12)
    assert np.allclose(dX, Xt.grad.numpy(), rtol=1e-10, atol=1e-12)
    for k in range(4):
        assert np.allclose(dW[k], Wt[k].grad.numpy(), rtol=1e-10, atol=1e-12), k


def test_network_rounding_points():
    rng = _rng(9)
    W = _weights()
    X = rng.normal(size=(256, 64))
    o, a = S.mlp_forward(X, W)
    o64, _ = S.mlp_forward(X, W, rounding=False)
    for k in range(4):
        assert np.array_equal(a[k], S.bf16(a[k]))                   # products see bf16 inputs
    rel = np.abs(o - o64) / (np.abs(o64).max())
    assert rel.max() < 3e-2 and rel.mean() < 4e-3                   # bf16 rounding of 4 inputs
    do = rng.normal(size=(256, 16))
    dX, dW = S.mlp_backward(a, W, do)
    dX64, _ = S.mlp_backward(a, W, do, rounding=False)
    assert np.abs(dX - dX64).max() < 3e-2 * np.abs(dX64).max()


def test_head_derivatives():
    rng = _rng(10)
    o = rng.normal(size=(100, 16)) * 2
    D = rng.uniform(0, 3, 100)
    K, k0, k1, v = S.head(o, D)
    h = 1e-6
    for j, ref in ((0, k0), (1, k1)):
        op, om = o.copy(), o.copy()
        op[:, j] += h
        om[:, j] -= h
        fd = (S.head(op, D)[0] - S.head(om, D)[0]) / (2 * h)
        assert np.allclose(ref, fd, rtol=1e-6, atol=1e-10)
    assert np.allclose(v, (S.head(o, D + h)[0] - S.head(o, D - h)[0]) / (2 * h), rtol=1e-6)


def _problem(seed=11, T=120, n_solves=3):
    rng = _rng(seed)
    x, nt = _texels(T, seed)
    area = rng.uniform(0.5, 1.5, T) * 0.01
    lo = np.array([-1.0, -1.0, -0.5], np.float32)
    ext = 8.0
    inv_ext = np.float32(1.0 / ext)
    lights = np.array([_spot(x=rng.uniform(1, 5), y=rng.uniform(1, 3), yaw=rng.uniform(0, 6), pitch=-1.3 + 0.2 * i)
                       for i in range(n_solves)])
    table = rng.normal(size=(16, S.TABLE, 2)) * 0.5
    W = _weights(seed, scale=0.3)
    return x.astype(np.float32), nt, area, lo, ext, inv_ext, lights, table, W


def test_training_gradients_against_central_differences():
    x, nt, area, lo, ext, inv_ext, lights, table, W = _problem()
    rng = _rng(12)
    samples = np.column_stack([rng.integers(0, 3, 200), rng.integers(0, x.shape[0], 200)])
    E_obs = rng.uniform(0, 0.3, size=(3, x.shape[0]))
    args = (samples, lights, E_obs, x, nt, area, lo, ext, inv_ext)
    loss, dW, dt = S.train_gradients(table, W, *args, rounding=False)
    h = 1e-6
    for k, (i, j) in ((0, (3, 40)), (1, (5, 7)), (2, (60, 2)), (3, (0, 11)), (3, (1, 30))):
        Wp = [w.copy() for w in W]
        Wm = [w.copy() for w in W]
        Wp[k][i, j] += h
        Wm[k][i, j] -= h
        fd = (S.train_gradients(table, Wp, *args, rounding=False)[0]
              - S.train_gradients(table, Wm, *args, rounding=False)[0]) / (2 * h)
        assert dW[k][i, j] == pytest.approx(fd, rel=1e-5, abs=1e-9), (k, i, j)
    nz = np.argwhere(np.abs(dt) > 1e-3 * np.abs(dt).max())
    for (l, e, f) in nz[:: max(1, len(nz) // 6)][:6]:
        tp, tm = table.copy(), table.copy()
        tp[l, e, f] += h
        tm[l, e, f] -= h
        fd = (S.train_gradients(tp, W, *args, rounding=False)[0]
              - S.train_gradients(tm, W, *args, rounding=False)[0]) / (2 * h)
        assert dt[l, e, f] == pytest.approx(fd, rel=1e-5, abs=1e-9), (l, e, f)


def test_design_gradient_against_central_differences():
    x, nt, area, lo, ext, inv_ext, lights, table, W = _problem(13, T=150, n_solves=2)
    lights = lights.copy()
    lights[:, 6] = [2.0, 1.5]
    rng = _rng(14)
    target = rng.uniform(0, 0.5, x.shape[0])
    alpha = rng.uniform(0.5, 1.0, x.shape[0])
    args = (x, nt, area, target, alpha, lo, ext, inv_ext)
    O, g, E = S.design_objective(table, W, lights, *args, rounding=False)
    assert g[:, 7].tolist() == [0.0, 0.0]
    for l in range(2):
        for k, c in enumerate([1, 2, 3, 4, 5, 6, 7]):
            h = 1e-6
            lp, lm = lights.copy(), lights.copy()
            lp[l, c] += h
            lm[l, c] -= h
            fd = (S.design_objective(table, W, lp, *args, rounding=False)[0]
                  - S.design_objective(table, W, lm, *args, rounding=False)[0]) / (2 * h)
            assert g[l, c - 1] == pytest.approx(fd, rel=2e-5, abs=1e-7 * abs(O)), (l, c)


def test_adam_matches_torch():
    rng = _rng(15)
    p0 = rng.normal(size=50)
    grads = [rng.normal(size=50) for _ in range(4)]
    pt = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.Adam([pt], lr=1e-2, betas=(0.9, 0.99), eps=1e-15)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for k, g in enumerate(grads):
        opt.zero_grad()
        pt.grad = torch.tensor(g)
        opt.step()
        p, m, v = S.adam(p, g, m, v, k + 1, 1e-2)
    assert np.allclose(p, pt.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_texel_centres_of_a_plane_and_a_box():
    sc = scenes.plane(half=1.0, res=8, albedo=0.5)
    pos, nrm = S.texel_centres(sc)
    lo = sc.xyz.reshape(-1, 3).min(0)
    hi = sc.xyz.reshape(-1, 3).max(0)
    # every centre lies in the plane, one per texel cell, on the cell centres
    assert np.allclose(np.abs(nrm[:, 2]), 1.0)
    span = hi - lo
    ax = [a for a in range(3) if span[a] > 0]
    cells = np.round((pos[:, ax] - lo[ax]) / span[ax] * 8 - 0.5, 9)
    assert np.allclose(cells, np.round(cells)) and len({tuple(c) for c in cells}) == 64
    # the oracle tracer's texel lookup sends a ray through each centre into that texel
    box = scenes.closed_cube(res=4, albedo=0.5)
    p2, n2 = S.texel_centres(box)
    centre = box.xyz.reshape(-1, 3).mean(0)
    org = np.repeat(centre[None], p2.shape[0], 0)
    d = p2 - org
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    tri, t, b = oracle.closest_hits(box, org, d)
    uv = box.uv[tri].astype(np.float64)
    u = np.einsum("ni,ni->n", b, uv[:, :, 0])
    v = np.einsum("ni,ni->n", b, uv[:, :, 1])
    tile = box.tile[tri]
    ru, rv = box.tile_res[tile, 0], box.tile_res[tile, 1]
    texel = box.texel_offsets()[tile] + np.floor(u * ru).astype(np.int64) + ru * np.floor(v * rv).astype(np.int64)
    assert np.array_equal(texel, np.arange(box.n_texels))
    assert np.allclose(np.abs(np.sum(n2 * (p2 - centre), axis=1)), 0.5)
