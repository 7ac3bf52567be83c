"""CPU oracle of the irradiance surrogate (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU leg
may import this module; the product path never does. Everything here is plain
numpy in float64, written to be read against the model's definition below,
with no blocking or fusion.

The surrogate predicts the irradiance a unit-intensity spot light puts on a
texel, K(t, l), so that a design's irradiance is the sum over its lights,
E_t = sum_l I_l K(t, l) (irradiance is linear in the emitted power and
additive over lights, Eq. 7-8 with I_e = p^2 / 2). K is split into the
unoccluded direct term D, which has a closed form (the inverse-square cosine
law of the point source of Sec. 4.4 times the spot falloff a(theta) of Eq.
S.11), and learned parts:

    K = sigmoid(o_0) * D + R_SCALE * softplus(o_1),   D = a(theta) |cos_r| / r^2

where o = MLP(x) is a 4-layer, 64-wide ReLU network without biases on a
64-wide input x: a 16-level multiresolution hash encoding of the texel centre
(Mueller et al., Instant neural graphics primitives, 2022: L = 16 levels,
F = 2 features per entry, 2^19 entries per level, spatial hash with the
primes 1, 2654435761, 805459861; dense indexing where a level's grid fits)
followed by geometric features of the light relative to the texel. The
weights are bf16 and every product is accumulated in fp32 on the GPU; the
inputs to every matrix product (x, hidden activations, back-propagated
gradients) are rounded to bf16. This oracle applies the same roundings at the
same points and accumulates in float64.

Input layout (x, 64 entries):
    0..31   hash encoding, level-major, 2 features per level
    32..34  u, the unit vector from the texel centre to the light
    35      r / 10 (r in metres)
    36..38  n_l, the spot axis
    39      cos_l = -u . n_l
    40      |cos_r| = |n_t . u|
    41      a(cos_l), the spot falloff
    42      cos(theta_in)
    43..45  (p - lo) / ext, the light position in the normalised scene box
    46..48  n_t, the texel normal
    49      1
    50..63  0

Training loss over a batch of (solve s, texel t) samples with observed
irradiance E_obs of a unit-intensity light:
    loss = (1 / B) sum_b 1/2 (A_t / A_mean) (K_b - E_obs_b)^2.
Design objective (Eq. 6 at order 0 with the surrogate's irradiance):
    O = 1/2 sum_t A_t alpha_t (E_t - E*_t)^2.
"""
from __future__ import annotations

import numpy as np

N_LEVELS = 16
N_FEAT = 2
LOG2_TABLE = 19
TABLE = 1 << LOG2_TABLE
# grid resolution of each level: floor(16 * 2^(l / 3)), 16 ... 512
RES = (16, 20, 25, 32, 40, 50, 64, 80, 101, 128, 161, 203, 256, 322, 406, 512)
PRIMES = (1, 2654435761, 805459861)
N_IN, N_HID, N_OUT = 64, 64, 16
R_SCALE = 0.01
F_U, F_R, F_NL, F_COSL, F_COSR, F_A, F_CIN, F_P, F_NT, F_ONE = 32, 35, 36, 39, 40, 41, 42, 43, 46, 49
N_GEOM = 17                  # entries 32..48 depend on the light and the texel
N_THETA = 6                  # x, y, z, yaw, pitch, theta_in
WEIGHT_SHAPES = ((N_HID, N_IN), (N_HID, N_HID), (N_HID, N_HID), (N_OUT, N_HID))


# ---------------------------------------------------------------------------
# rounding
# ---------------------------------------------------------------------------
def bf16(x):
    """Round to bfloat16 (returned as float64): first to float32, then to the
    nearest bfloat16, ties to even (the kernel rounds its float32 values)."""
    f = np.asarray(x, np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    b = (b + np.uint64(0x7FFF) + lsb) >> np.uint64(16) << np.uint64(16)
    out = (b & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if np.any(nan):
        out = np.where(nan, np.nan, out)
    return out


# ---------------------------------------------------------------------------
# multiresolution hash encoding
# ---------------------------------------------------------------------------
def normalise(x, lo, inv_ext):
    """Position in the normalised box, float32 arithmetic (the kernel's: the
    grid cell is an integer decision): (x - lo) * inv_ext, each op rounded."""
    x32 = np.asarray(x, np.float32)
    return ((x32 - np.asarray(lo, np.float32)).astype(np.float32) * np.float32(inv_ext)).astype(np.float32)


def dense_level(level: int) -> bool:
    n = RES[level] + 1
    return n * n * n <= TABLE


def vertex_index(level: int, v):
    """Table slot of integer grid vertices v [..., 3] (int64) of a level:
    x + (N+1)(y + (N+1) z) where the grid fits, else the spatial hash
    (x*1 xor y*2654435761 xor z*805459861) mod 2^19 in 32-bit arithmetic."""
    v = np.asarray(v, np.int64)
    if dense_level(level):
        n = RES[level] + 1
        return v[..., 0] + n * (v[..., 1] + n * v[..., 2])
    h = np.zeros(v.shape[:-1], np.uint64)
    for a in range(3):
        h ^= (v[..., a].astype(np.uint64) * np.uint64(PRIMES[a])) & np.uint64(0xFFFFFFFF)
    return (h & np.uint64(TABLE - 1)).astype(np.int64)


def _cells(xn32, level):
    """Lower grid vertex and float32 fractional position of each point."""
    n = np.float32(RES[level])
    pos = (xn32 * n).astype(np.float32)
    i0 = np.floor(pos).astype(np.int64)
    i0 = np.clip(i0, 0, RES[level] - 1)
    f = (pos - i0.astype(np.float32)).astype(np.float32).astype(np.float64)
    return i0, np.clip(f, 0.0, 1.0)


CORNERS = np.array([[(c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], np.int64)


def corner_weights(f):
    """Trilinear weights of the 8 corners, [B, 8]; corner c has offset bits
    (x, y, z) = (c & 1, c >> 1 & 1, c >> 2 & 1)."""
    w = np.ones(f.shape[:-1] + (8,))
    for c in range(8):
        for a in range(3):
            w[..., c] *= f[..., a] if CORNERS[c, a] else 1.0 - f[..., a]
    return w


def encode(xn32, table):
    """Hash encoding [B, 32] of normalised positions xn32 [B, 3] (float32)
    with table [16, 2^19, 2]: per level the trilinear interpolation of the
    features stored at the 8 corners of the point's grid cell."""
    xn32 = np.asarray(xn32, np.float32).reshape(-1, 3)
    out = np.zeros((xn32.shape[0], N_LEVELS * N_FEAT))
    for l in range(N_LEVELS):
        i0, f = _cells(xn32, l)
        w = corner_weights(f)
        for c in range(8):
            idx = vertex_index(l, i0 + CORNERS[c])
            out[:, 2 * l:2 * l + 2] += w[:, c:c + 1] * table[l, idx, :]
    return out


def encode_backward(xn32, g):
    """Gradient of sum(g * encode(xn32, table)) with respect to the table
    (the encoding is linear in the table)."""
    xn32 = np.asarray(xn32, np.float32).reshape(-1, 3)
    dt = np.zeros((N_LEVELS, TABLE, N_FEAT))
    for l in range(N_LEVELS):
        i0, f = _cells(xn32, l)
        w = corner_weights(f)
        for c in range(8):
            idx = vertex_index(l, i0 + CORNERS[c])
            for j in range(N_FEAT):
                np.add.at(dt[l, :, j], idx, w[:, c] * g[:, 2 * l + j])
    return dt


# ---------------------------------------------------------------------------
# geometric light features and their derivatives
# ---------------------------------------------------------------------------
def spot_axis(yaw, pitch):
    """n(yaw, pitch) = (cos p cos y, cos p sin y, sin p) and its derivatives."""
    cy, sy, cp, sp = np.cos(yaw), np.sin(yaw), np.cos(pitch), np.sin(pitch)
    n = np.array([cp * cy, cp * sy, sp])
    dn_dyaw = np.array([-cp * sy, cp * cy, 0.0])
    dn_dpitch = np.array([-sp * cy, -sp * sy, cp])
    return n, dn_dyaw, dn_dpitch


def falloff(cos_l, theta_in, theta_out):
    """Spot falloff a (Eq. S.11): 1 inside the inner cone, ((cos - cos_out) /
    (cos_in - cos_out))^2 between the cones, 0 outside; with da/dcos and
    da/dtheta_in."""
    ci, co = np.cos(theta_in), np.cos(theta_out)
    cos_l = np.asarray(cos_l, np.float64)
    s = (cos_l - co) / (ci - co)
    soft = (cos_l > co) & (cos_l < ci)
    a = np.where(cos_l >= ci, 1.0, np.where(soft, s * s, 0.0))
    da_dcos = np.where(soft, 2.0 * s / (ci - co), 0.0)
    da_dci = np.where(soft, -2.0 * s * s / (ci - co), 0.0)
    return a, da_dcos, da_dci * (-np.sin(theta_in))


def geometry(light, x, n_t, lo, ext):
    """Entries 32..48 of the input for one light (row of the light array:
    type, x, y, z, yaw, pitch, p_int, theta_in, theta_out) and texel centres
    x [B, 3] with normals n_t [B, 3]; the direct term D; and their derivatives
    with respect to theta = (x, y, z, yaw, pitch, theta_in):
    returns G [B, 17], dG [B, 17, 6], D [B], dD [B, 6]."""
    p = np.asarray(light[1:4], np.float64)
    yaw, pitch, th_in, th_out = float(light[4]), float(light[5]), float(light[7]), float(light[8])
    x = np.asarray(x, np.float64).reshape(-1, 3)
    n_t = np.asarray(n_t, np.float64).reshape(-1, 3)
    B = x.shape[0]
    d = p[None, :] - x
    r = np.linalg.norm(d, axis=1)
    u = d / r[:, None]
    P = (np.eye(3)[None] - u[:, :, None] * u[:, None, :]) / r[:, None, None]    # du/dp
    nl, dn_y, dn_p = spot_axis(yaw, pitch)
    cos_l = -u @ nl
    cr = np.sum(n_t * u, axis=1)
    sgn = np.sign(cr)
    a, da_dcos, da_dthin = falloff(cos_l, th_in, th_out)

    G = np.zeros((B, N_GEOM))
    dG = np.zeros((B, N_GEOM, N_THETA))
    k = lambda f: f - F_U                                                         # noqa: E731
    G[:, k(F_U):k(F_U) + 3] = u
    dG[:, k(F_U):k(F_U) + 3, 0:3] = P
    G[:, k(F_R)] = r / 10.0
    dG[:, k(F_R), 0:3] = u / 10.0
    G[:, k(F_NL):k(F_NL) + 3] = nl[None, :]
    dG[:, k(F_NL):k(F_NL) + 3, 3] = dn_y[None, :]
    dG[:, k(F_NL):k(F_NL) + 3, 4] = dn_p[None, :]
    G[:, k(F_COSL)] = cos_l
    dcosl = np.zeros((B, N_THETA))
    dcosl[:, 0:3] = -np.einsum("bij,j->bi", P, nl)
    dcosl[:, 3] = -u @ dn_y
    dcosl[:, 4] = -u @ dn_p
    dG[:, k(F_COSL)] = dcosl
    G[:, k(F_COSR)] = np.abs(cr)
    dcosr = np.zeros((B, N_THETA))
    dcosr[:, 0:3] = sgn[:, None] * np.einsum("bij,bj->bi", P, n_t)
    dG[:, k(F_COSR)] = dcosr
    G[:, k(F_A)] = a
    da = da_dcos[:, None] * dcosl
    da[:, 5] += da_dthin
    dG[:, k(F_A)] = da
    G[:, k(F_CIN)] = np.cos(th_in)
    dG[:, k(F_CIN), 5] = -np.sin(th_in)
    G[:, k(F_P):k(F_P) + 3] = ((p - np.asarray(lo, np.float64)) / ext)[None, :]
    dG[:, k(F_P):k(F_P) + 3, 0:3] = np.eye(3)[None] / ext
    G[:, k(F_NT):k(F_NT) + 3] = n_t

    D = a * np.abs(cr) / (r * r)
    dD = da * (np.abs(cr) / (r * r))[:, None] + dcosr * (a / (r * r))[:, None]
    dD[:, 0:3] += (-2.0 * a * np.abs(cr) / r ** 3)[:, None] * u
    return G, dG, D, dD


def inputs(enc, G):
    """The 64-entry input rows (float64, before the bf16 rounding)."""
    B = enc.shape[0]
    X = np.zeros((B, N_IN))
    X[:, 0:32] = enc
    X[:, F_U:F_U + N_GEOM] = G
    X[:, F_ONE] = 1.0
    return X


# ---------------------------------------------------------------------------
# the network
# ---------------------------------------------------------------------------
def _round(x, rounding):
    return bf16(x) if rounding else np.asarray(x, np.float64)


def mlp_forward(X, W, rounding=True):
    """o = W3 relu(W2 relu(W1 relu(W0 x))) with bf16 inputs to every product.
    W: four bf16-valued float64 arrays [out, in]. Returns the output [B, 16]
    and the cache (bf16 inputs a0..a3 of the four products). rounding=False
    gives the same network in plain float64."""
    a = [_round(X, rounding)]
    for k in range(3):
        z = a[k] @ W[k].T
        a.append(_round(np.maximum(z, 0.0), rounding))
    o = a[3] @ W[3].T
    return o, a


def mlp_backward(a, W, do, rounding=True):
    """Back-propagation of do = dloss/do [B, 16]: the gradient reaching each
    product is rounded to bf16 before it is multiplied. Returns dX [B, 64]
    (gradient at the input) and dW (four arrays, summed over the rows)."""
    dz = _round(do, rounding)
    dW = [None] * 4
    for k in (3, 2, 1, 0):
        dW[k] = dz.T @ a[k]
        da = dz @ W[k]
        if k == 0:
            return da, dW
        dz = _round(da * (a[k] > 0.0), rounding)
    raise AssertionError


def sigmoid(v):
    return 1.0 / (1.0 + np.exp(-v))


def head(o, D):
    """K = sigmoid(o0) D + R_SCALE softplus(o1), and dK/do0, dK/do1, dK/dD."""
    v = sigmoid(o[:, 0])
    sp = np.logaddexp(0.0, o[:, 1])
    K = v * D + R_SCALE * sp
    return K, v * (1.0 - v) * D, R_SCALE * sigmoid(o[:, 1]), v


# ---------------------------------------------------------------------------
# whole evaluations
# ---------------------------------------------------------------------------
def response(table, W, light, x, n_t, lo, ext, inv_ext, rounding=True):
    """K(t, light) for texel centres x [B, 3] (float32 values), normals n_t."""
    enc = encode(normalise(x, lo, inv_ext), table)
    G, _, D, _ = geometry(light, x, n_t, lo, ext)
    o, _ = mlp_forward(inputs(enc, G), W, rounding)
    return head(o, D)[0]


def train_gradients(table, W, samples, lights, E_obs, x, n_t, area, lo, ext, inv_ext, rounding=True):
    """Loss and gradients of one training batch. samples [B, 2] = (solve s,
    texel t); lights [S, 9] the unit-intensity light of every solve; E_obs
    [S, T] the observed irradiance; x, n_t, area per texel. Returns (loss,
    dW (4 arrays), dtable [16, 2^19, 2])."""
    s, t = samples[:, 0], samples[:, 1]
    B = samples.shape[0]
    xt = np.asarray(x, np.float32)[t]
    enc = encode(normalise(xt, lo, inv_ext), table)
    G = np.zeros((B, N_GEOM))
    D = np.zeros(B)
    for si in np.unique(s):
        m = s == si
        g, _, d, _ = geometry(lights[si], xt[m], n_t[t[m]], lo, ext)
        G[m], D[m] = g, d
    o, cache = mlp_forward(inputs(enc, G), W, rounding)
    K, dK_do0, dK_do1, _ = head(o, D)
    wgt = np.asarray(area, np.float64)[t] / float(np.mean(area))
    e = K - np.asarray(E_obs, np.float64)[s, t]
    loss = float(np.sum(0.5 * wgt * e * e) / B)
    dK = wgt * e / B
    do = np.zeros((B, N_OUT))
    do[:, 0] = dK * dK_do0
    do[:, 1] = dK * dK_do1
    dX, dW = mlp_backward(cache, W, do, rounding)
    dtable = encode_backward(normalise(xt, lo, inv_ext), dX[:, 0:32])
    return loss, dW, dtable


def design_objective(table, W, lights, x, n_t, area, target, alpha, lo, ext, inv_ext, rounding=True):
    """O = 1/2 sum_t A_t alpha_t (E_t - E*_t)^2 with E_t = sum_l I_l K(t, l),
    I_l = p_l^2 / 2, and dO/dp [L, 8] in the order (x, y, z, yaw, pitch,
    p_int, theta_in, theta_out); theta_out gets no gradient (the surrogate is
    trained at a fixed outer cone). Returns (O, grad, E)."""
    x32 = np.asarray(x, np.float32)
    enc = encode(normalise(x32, lo, inv_ext), table)
    L = lights.shape[0]
    T = x32.shape[0]
    Ks, caches = [], []
    E = np.zeros(T)
    for l in range(L):
        G, dG, D, dD = geometry(lights[l], x32, n_t, lo, ext)
        o, cache = mlp_forward(inputs(enc, G), W, rounding)
        K, dK_do0, dK_do1, v = head(o, D)
        Ks.append(K)
        caches.append((cache, dG, dD, dK_do0, dK_do1, v))
        E += 0.5 * lights[l, 6] ** 2 * K
    w = np.asarray(alpha, np.float64) * (E - np.asarray(target, np.float64))
    A = np.asarray(area, np.float64)
    O = float(0.5 * np.sum(A * w * (E - np.asarray(target, np.float64))))
    grad = np.zeros((L, 8))
    for l in range(L):
        cache, dG, dD, dK_do0, dK_do1, v = caches[l]
        I = 0.5 * lights[l, 6] ** 2
        up = A * w * I                        # dO/dK_tl
        do = np.zeros((T, N_OUT))
        do[:, 0] = up * dK_do0
        do[:, 1] = up * dK_do1
        dX, _ = mlp_backward(cache, W, do, rounding)
        dth = np.einsum("bg,bgk->k", dX[:, F_U:F_U + N_GEOM], dG) + np.einsum("b,bk->k", up * v, dD)
        grad[l, 0:5] = dth[0:5]
        grad[l, 6] = dth[5]
        grad[l, 5] = np.sum(A * w * Ks[l]) * lights[l, 6]
    return O, grad, E


def adam(param, grad, m, v, step, lr, beta1=0.9, beta2=0.99, eps=1e-15):
    """One Adam step (Kingma and Ba 2015) with bias correction; step counts
    from 1. Returns (param, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return param - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------------------
# texel centres
# ---------------------------------------------------------------------------
def texel_centres(scene):
    """World position and unit normal of every texel centre: the point of the
    tile whose chart coordinates are ((i + 1/2) / res_u, (j + 1/2) / res_v),
    mapped through the barycentric coordinates of the tile triangle that
    contains it in the chart (the one whose smallest barycentric coordinate is
    largest, clamped to the triangle when none contains it)."""
    T = scene.n_texels
    off = scene.texel_offsets()
    pos = np.zeros((T, 3))
    nrm = np.zeros((T, 3))
    tris_of = [[] for _ in range(scene.n_tiles)]
    for i, k in enumerate(scene.tile):
        tris_of[int(k)].append(i)
    for k in range(scene.n_tiles):
        ru, rv = int(scene.tile_res[k, 0]), int(scene.tile_res[k, 1])
        iv, iu = np.meshgrid(np.arange(rv), np.arange(ru), indexing="ij")
        q = np.stack([(iu.ravel() + 0.5) / ru, (iv.ravel() + 0.5) / rv], axis=1)
        best = np.full(q.shape[0], -np.inf)
        for tri in tris_of[k]:
            uv = scene.uv[tri].astype(np.float64)
            X = scene.xyz[tri].astype(np.float64)
            e1, e2 = uv[1] - uv[0], uv[2] - uv[0]
            det = e1[0] * e2[1] - e1[1] * e2[0]
            dq = q - uv[0]
            b1 = (dq[:, 0] * e2[1] - dq[:, 1] * e2[0]) / det
            b2 = (e1[0] * dq[:, 1] - e1[1] * dq[:, 0]) / det
            b0 = 1.0 - b1 - b2
            score = np.minimum(np.minimum(b0, b1), b2)
            take = score > best
            b = np.clip(np.stack([b0, b1, b2], axis=1), 0.0, None)
            b /= b.sum(axis=1, keepdims=True)
            n = np.cross(X[1] - X[0], X[2] - X[0])
            n /= np.linalg.norm(n)
            pos[off[k]:off[k + 1]][take] = (b @ X)[take]
            nrm[off[k]:off[k + 1]][take] = n
            best = np.where(take, score, best)
    return pos, nrm
