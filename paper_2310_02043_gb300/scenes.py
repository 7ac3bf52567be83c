"""Seeded synthetic inputs: scenes, luminaires and their perturbations.

This module is the one place both the CUDA path and the CPU oracle take their
inputs from. It builds geometry and parameter arrays only; it holds none of the
light-transport arithmetic (no flux, no sampling, no intersection, no texel
lookup), so that the two implementations stay independent.

Scene layout (all arrays are C-contiguous numpy):

* ``xyz``       float32 [n_tri, 3, 3]  triangle vertex positions, metres
* ``uv``        float32 [n_tri, 3, 2]  per-vertex coordinates in the triangle's
                                       tile chart, in [0, 1]^2
* ``tile``      int32   [n_tri]        tile (texel chart) of each triangle
* ``albedo``    float32 [n_tri]        Lambertian albedo rho in [0, 1]
* ``tile_res``  int32   [n_tiles, 2]   texel resolution (res_u, res_v)
* ``tile_area`` float64 [n_tiles]      surface area the tile covers, m^2

A planar quad is one tile made of two triangles that share the quad's chart;
a lone triangle is a 1x1 tile. Texels of a tile are numbered
``u_index + res_u * v_index`` after all texels of the tiles before it.

Luminaires are a float64 array [n_lights, 9] with columns ``LIGHT_FIELDS``:
type (0 point, 1 spot), position x, y, z, yaw, pitch (radians; the spot axis
is (cos p cos y, cos p sin y, sin p) with z up), p_int (the intensity
parameter, I_e = p_int^2 / 2 as in Sec. 4.4.1 of the paper), theta_in and
theta_out (spot cone half-angles, radians).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

LIGHT_FIELDS = ("type", "x", "y", "z", "yaw", "pitch", "p_int", "theta_in", "theta_out")
POINT, SPOT, AREA = 0, 1, 2
GRAD_FIELDS = ("x", "y", "z", "yaw", "pitch", "p_int", "theta_in", "theta_out")


@dataclass
class Scene:
    name: str
    xyz: np.ndarray
    uv: np.ndarray
    tile: np.ndarray
    albedo: np.ndarray
    tile_res: np.ndarray
    tile_area: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n_tri(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_tiles(self) -> int:
        return int(self.tile_res.shape[0])

    @property
    def n_texels(self) -> int:
        return int(np.sum(self.tile_res[:, 0].astype(np.int64) * self.tile_res[:, 1]))

    def texel_offsets(self) -> np.ndarray:
        """First texel index of every tile, plus the total at the end."""
        counts = self.tile_res[:, 0].astype(np.int64) * self.tile_res[:, 1]
        return np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)

    def bbox_diagonal(self) -> float:
        pts = self.xyz.reshape(-1, 3).astype(np.float64)
        return float(np.linalg.norm(pts.max(0) - pts.min(0)))


class _Builder:
    """Accumulates quads and triangles into the flat scene arrays."""

    def __init__(self):
        self.xyz, self.uv, self.tile, self.albedo = [], [], [], []
        self.res, self.area = [], []

    def quad(self, corner, a, b, res_u, res_v, albedo):
        """Parallelogram corner + s*a + t*b, s, t in [0, 1]; one tile."""
        c = np.asarray(corner, np.float64)
        a = np.asarray(a, np.float64)
        b = np.asarray(b, np.float64)
        t = len(self.res)
        p00, p10, p11, p01 = c, c + a, c + a + b, c + b
        self.xyz += [[p00, p10, p11], [p00, p11, p01]]
        self.uv += [[[0, 0], [1, 0], [1, 1]], [[0, 0], [1, 1], [0, 1]]]
        self.tile += [t, t]
        self.albedo += [albedo, albedo]
        self.res.append([int(res_u), int(res_v)])
        self.area.append(float(np.linalg.norm(np.cross(a, b))))

    def quad_pitch(self, corner, a, b, pitch, albedo):
        """Quad whose texel count follows a target texel pitch (metres)."""
        ru = max(1, int(np.ceil(np.linalg.norm(a) / pitch - 1e-9)))
        rv = max(1, int(np.ceil(np.linalg.norm(b) / pitch - 1e-9)))
        self.quad(corner, a, b, ru, rv, albedo)

    def triangle(self, p0, p1, p2, albedo):
        """A lone triangle is a 1x1 tile."""
        p0, p1, p2 = (np.asarray(p, np.float64) for p in (p0, p1, p2))
        t = len(self.res)
        self.xyz.append([p0, p1, p2])
        self.uv.append([[0, 0], [1, 0], [0, 1]])
        self.tile.append(t)
        self.albedo.append(albedo)
        self.res.append([1, 1])
        self.area.append(0.5 * float(np.linalg.norm(np.cross(p1 - p0, p2 - p0))))

    def box(self, lo, hi, res_or_pitch, albedo, faces=("-x", "+x", "-y", "+y", "-z", "+z"), pitch=False):
        lo = np.asarray(lo, np.float64)
        hi = np.asarray(hi, np.float64)
        dx, dy, dz = hi - lo
        ex, ey, ez = np.array([dx, 0, 0]), np.array([0, dy, 0]), np.array([0, 0, dz])
        spec = {
            "-x": (lo, ey, ez),
            "+x": (lo + ex, ey, ez),
            "-y": (lo, ex, ez),
            "+y": (lo + ey, ex, ez),
            "-z": (lo, ex, ey),
            "+z": (lo + ez, ex, ey),
        }
        for f in faces:
            c, a, b = spec[f]
            if pitch:
                self.quad_pitch(c, a, b, res_or_pitch, albedo)
            else:
                self.quad(c, a, b, res_or_pitch, res_or_pitch, albedo)

    def build(self, name, **meta) -> Scene:
        return Scene(
            name=name,
            xyz=np.ascontiguousarray(np.asarray(self.xyz, np.float32)),
            uv=np.ascontiguousarray(np.asarray(self.uv, np.float32)),
            tile=np.ascontiguousarray(np.asarray(self.tile, np.int32)),
            albedo=np.ascontiguousarray(np.asarray(self.albedo, np.float32)),
            tile_res=np.ascontiguousarray(np.asarray(self.res, np.int32).reshape(-1, 2)),
            tile_area=np.ascontiguousarray(np.asarray(self.area, np.float64)),
            meta=dict(meta),
        )


def make_lights(rows) -> np.ndarray:
    """Rows of (type, x, y, z, yaw, pitch, p_int, theta_in, theta_out)."""
    arr = np.asarray(rows, np.float64).reshape(-1, len(LIGHT_FIELDS))
    return np.ascontiguousarray(arr)


def point_light(pos, intensity):
    """Point light with I_e = intensity (p_int = sqrt(2 I_e))."""
    return [POINT, *pos, 0.0, 0.0, float(np.sqrt(2.0 * intensity)), 0.0, 0.0]


def spot_light(pos, yaw, pitch, intensity, theta_in, theta_out):
    return [SPOT, *pos, yaw, pitch, float(np.sqrt(2.0 * intensity)), theta_in, theta_out]


def area_light(pos, yaw, pitch, power, width, height):
    """Rectangular Lambertian area light centred at pos, normal n(yaw, pitch),
    edges along dn/dpitch (width) and n x dn/dpitch (height), total emitted
    power P (p_int = sqrt(2 P)); the width and height take the theta_in and
    theta_out slots of the row."""
    return [AREA, *pos, yaw, pitch, float(np.sqrt(2.0 * power)), width, height]


# --------------------------------------------------------------------------
# Workload scenes
# --------------------------------------------------------------------------

def cornell_box(res: int = 32, albedo: float = 0.7) -> Scene:
    """Cornell-box room: 1 m cube with the front (y = 0) open, 5 room quads,
    a short 0.3 m box and a tall 0.3 x 0.3 x 0.6 m box without bottoms (they
    rest on the floor). 15 quads = 30 triangles, res x res texels per face."""
    b = _Builder()
    one = 1.0
    b.quad([0, 0, 0], [one, 0, 0], [0, one, 0], res, res, albedo)      # floor z = 0
    b.quad([0, 0, one], [one, 0, 0], [0, one, 0], res, res, albedo)    # ceiling z = 1
    b.quad([0, one, 0], [one, 0, 0], [0, 0, one], res, res, albedo)    # back wall y = 1
    b.quad([0, 0, 0], [0, one, 0], [0, 0, one], res, res, albedo)      # left wall x = 0
    b.quad([one, 0, 0], [0, one, 0], [0, 0, one], res, res, albedo)    # right wall x = 1
    sides = ("-x", "+x", "-y", "+y", "+z")
    b.box([0.2, 0.55, 0.0], [0.5, 0.85, 0.3], res, albedo, faces=sides)
    b.box([0.55, 0.25, 0.0], [0.85, 0.55, 0.6], res, albedo, faces=sides)
    return b.build("cornell", res=res, albedo=albedo)


def cornell_lights() -> np.ndarray:
    """One point light at (0.5, 0.5, 0.9), I_e = 1."""
    return make_lights([point_light((0.5, 0.5, 0.9), 1.0)])


def office(seed: int = 0, pitch: float = 0.02, n_boxes: int = 200) -> Scene:
    """Procedural office, 20 x 10 x 3 m closed room with ``n_boxes`` desks and
    cabinets (6 faces each, lifted 1 cm off the floor), texel pitch ``pitch``.

    Boxes sit one per cell of a 20 x 10 grid of 1 m cells (cells drawn without
    replacement when fewer than 200), jittered inside the cell: 60 % desks of
    0.9 x 0.7 x 0.75 m, 40 % cabinets of 0.5 x 0.45 x U[1, 2] m, each turned by
    0 or 90 degrees. Albedo is U[0.3, 0.8] per box and per room face."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    L, W, H = 20.0, 10.0, 3.0
    room = [
        ([0, 0, 0], [L, 0, 0], [0, W, 0]),   # floor
        ([0, 0, H], [L, 0, 0], [0, W, 0]),   # ceiling
        ([0, 0, 0], [L, 0, 0], [0, 0, H]),   # wall y = 0
        ([0, W, 0], [L, 0, 0], [0, 0, H]),   # wall y = W
        ([0, 0, 0], [0, W, 0], [0, 0, H]),   # wall x = 0
        ([L, 0, 0], [0, W, 0], [0, 0, H]),   # wall x = L
    ]
    for c, a, bb in room:
        b.quad_pitch(c, a, bb, pitch, float(rng.uniform(0.3, 0.8)))
    cells = rng.permutation(200)[:n_boxes]
    for cell in np.sort(cells):
        cx, cy = float(cell % 20), float(cell // 20)
        if rng.uniform() < 0.6:
            sx, sy, sz = 0.9, 0.7, 0.75
        else:
            sx, sy, sz = 0.5, 0.45, float(rng.uniform(1.0, 2.0))
        if rng.uniform() < 0.5:
            sx, sy = sy, sx
        margin = 0.05
        x0 = cx + margin + rng.uniform(0.0, 1.0 - 2 * margin - sx)
        y0 = cy + margin + rng.uniform(0.0, 1.0 - 2 * margin - sy)
        z0 = 0.01
        b.box([x0, y0, z0], [x0 + sx, y0 + sy, z0 + sz], pitch, float(rng.uniform(0.3, 0.8)), pitch=True)
    return b.build("office", seed=seed, pitch=pitch, n_boxes=n_boxes)


def office_lights(seed: int = 0, intensity: float = 50.0, theta_in_deg: float = 40.0,
                  theta_out_deg: float = 60.0) -> np.ndarray:
    """16 spots on a 4 x 4 grid at z = 2.8 m pointing down, pitch
    -pi/2 + U(-0.2, 0.2), yaw U(0, 2 pi)."""
    rng = np.random.default_rng(seed + 1000)
    rows = []
    for iy in range(4):
        for ix in range(4):
            x = 2.5 + 5.0 * ix
            y = 1.25 + 2.5 * iy
            yaw = float(rng.uniform(0.0, 2 * np.pi))
            pitch = -np.pi / 2 + float(rng.uniform(-0.2, 0.2))
            rows.append(spot_light((x, y, 2.8), yaw, pitch, intensity,
                                   np.radians(theta_in_deg), np.radians(theta_out_deg)))
    return make_lights(rows)


def office_designs(seed: int = 0, n_designs: int = 64, min_spots: int = 4, max_spots: int = 32,
                   total_intensity: float = 800.0, theta_in_deg: float = 40.0, theta_out_deg: float = 60.0):
    """Candidate lighting designs for the office: design d has n_d ~ U{min_spots
    .. max_spots} spots at z = 2.8 m, uniform over the 20 x 10 m ceiling (0.5 m
    from the walls), pitch -pi/2 + U(-0.2, 0.2), yaw U(0, 2 pi), and I_e =
    total_intensity / n_d each (every design emits the same power as the 16
    spots of office_lights). Returns (counts int32 [D], lights [sum n_d, 9])
    with the designs concatenated in order."""
    rng = np.random.default_rng(seed + 5000)
    counts = rng.integers(min_spots, max_spots + 1, size=n_designs).astype(np.int32)
    rows = []
    for n in counts:
        for _ in range(int(n)):
            x = float(rng.uniform(0.5, 19.5))
            y = float(rng.uniform(0.5, 9.5))
            yaw = float(rng.uniform(0.0, 2 * np.pi))
            pitch = -np.pi / 2 + float(rng.uniform(-0.2, 0.2))
            rows.append(spot_light((x, y, 2.8), yaw, pitch, total_intensity / int(n),
                                   np.radians(theta_in_deg), np.radians(theta_out_deg)))
    return counts, make_lights(rows)


def perturb_lights(lights: np.ndarray, seed: int, pos_sigma: float = 0.05, angle_sigma: float = 0.0,
                   intensity_range=(0.8, 1.2), theta_in_delta: float = 0.0) -> np.ndarray:
    """Seeded perturbation of a light array (the 'ground-truth' lights a target
    is traced from). Intensity I_e is scaled by U[intensity_range]."""
    rng = np.random.default_rng(seed)
    out = np.array(lights, np.float64, copy=True)
    n = out.shape[0]
    out[:, 1:4] += rng.normal(0.0, pos_sigma, size=(n, 3))
    if angle_sigma > 0:
        out[:, 4:6] += rng.normal(0.0, angle_sigma, size=(n, 2))
    scale = rng.uniform(intensity_range[0], intensity_range[1], size=n)
    out[:, 6] *= np.sqrt(scale)          # I_e = p^2 / 2 scales by `scale`
    if theta_in_delta > 0:
        spot = out[:, 0] == SPOT
        d = rng.uniform(-theta_in_delta, theta_in_delta, size=n)
        out[spot, 7] = np.minimum(out[spot, 7] + d[spot], out[spot, 8] - 1e-3)
    return np.ascontiguousarray(out)


# --------------------------------------------------------------------------
# Small scenes used to pin the oracle and to probe edge cases
# --------------------------------------------------------------------------

def plane(half: float = 1.0, res: int = 16, albedo: float = 0.5, z: float = 0.0) -> Scene:
    """A single square quad [-half, half]^2 at height z, res x res texels."""
    b = _Builder()
    b.quad([-half, -half, z], [2 * half, 0, 0], [0, 2 * half, 0], res, res, albedo)
    return b.build("plane", half=half, res=res)


def occluded_plane(half: float = 1.5, res: int = 8, occ_z: float = 0.4, occ_centre=(0.1, 0.0),
                   occ_half: float = 0.25, albedo: float = 0.5) -> Scene:
    """The plane z = 0 over [-half, half]^2 (res x res texels, the first
    res^2 texels) under a horizontal square occluder of half size occ_half
    centred at (occ_centre, occ_z) (2 x 2 texels): a light above casts a
    shadow whose outline moves with it."""
    b = _Builder()
    b.quad([-half, -half, 0.0], [2 * half, 0, 0], [0, 2 * half, 0], res, res, albedo)
    cx, cy = occ_centre
    b.quad([cx - occ_half, cy - occ_half, occ_z], [2 * occ_half, 0, 0], [0, 2 * occ_half, 0], 2, 2, albedo)
    return b.build("occluded_plane", half=half, res=res, occ_z=occ_z, occ_centre=tuple(occ_centre),
                   occ_half=occ_half)


def closed_cube(size: float = 1.0, res: int = 8, albedo: float = 0.5) -> Scene:
    """Closed cube [0, size]^3, 6 quads, uniform albedo (no ray escapes)."""
    b = _Builder()
    b.box([0, 0, 0], [size, size, size], res, albedo)
    return b.build("cube", size=size, res=res, albedo=albedo)


def icosphere(radius: float = 1.0, subdiv: int = 3, albedo: float = 0.5) -> Scene:
    """Closed icosphere centred at the origin; each triangle is a 1x1 tile."""
    t = (1.0 + 5 ** 0.5) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
             (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
             (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
             (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    v = [np.asarray(p, np.float64) / np.linalg.norm(p) for p in verts]
    for _ in range(subdiv):
        cache = {}

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = v[i] + v[j]
                v.append(m / np.linalg.norm(m))
                cache[key] = len(v) - 1
            return cache[key]

        nf = []
        for a, bb, c in faces:
            ab, bc, ca = mid(a, bb), mid(bb, c), mid(c, a)
            nf += [(a, ab, ca), (bb, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    b = _Builder()
    for a, bb, c in faces:
        b.triangle(radius * v[a], radius * v[bb], radius * v[c], albedo)
    return b.build("icosphere", radius=radius, subdiv=subdiv, albedo=albedo)


NESTED_SHELF_APEX = (0.0, 0.5, 0.0)


def nested_shelf(n_strips: int = 100, res: int = 8, strip_res: int = 2, albedo: float = 0.6) -> Scene:
    """A closed box room [-1, 2] x [-0.5, 1.5] x [-0.3, 1] (res x res texels
    per face) around a shelf of n_strips strips in the plane z = 0: strip i
    covers x in [2^-(i+1), 2^-i], y in [0.2, 0.8]. The strips halve in width
    towards NESTED_SHELF_APEX, so the surface-area heuristic peels them off
    one at a time and the 8-wide BVH has more than 8 levels while holding a
    few dozen nodes (small enough to stage in shared memory). A light at the
    apex lies in the strips' plane: every ray it emits starts inside the
    padded boxes of the whole chain, so it descends every level, and leaves
    the plane at t = 0, so it hits no strip."""
    b = _Builder()
    b.box([-1.0, -0.5, -0.3], [2.0, 1.5, 1.0], res, albedo)
    for i in range(n_strips):
        w = 0.5 ** (i + 1)
        b.quad([w, 0.2, 0.0], [w, 0.0, 0.0], [0.0, 0.6, 0.0], strip_res, strip_res, albedo)
    return b.build("nested_shelf", n_strips=n_strips, res=res)


def random_triangles(n: int, seed: int, extent: float = 1.0, albedo: float = 0.5) -> Scene:
    """n random triangles in [0, extent]^3 (a tiny scene for brute-force checks)."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    for _ in range(n):
        c = rng.uniform(0.1, 0.9, size=3) * extent
        p = [c + rng.normal(0, 0.2 * extent, size=3) for _ in range(3)]
        b.triangle(p[0], p[1], p[2], albedo)
    return b.build("random_triangles", seed=seed, n=n)


def random_rays(n: int, seed: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """n ray origins uniform in the box [lo, hi] and isotropic directions."""
    rng = np.random.default_rng(seed)
    o = rng.uniform(lo, hi, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o, d


def random_weights(n_texels: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded per-texel adjoint weights (used to inject dO/dE directly)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.normal(0.0, scale, size=n_texels).astype(np.float32))


# --------------------------------------------------------------------------
# Initial parameters of the irradiance surrogate
# --------------------------------------------------------------------------
def surrogate_init(seed: int = 0):
    """Seeded initial parameters of the irradiance surrogate: the four weight
    matrices ([64, 64] x 3 and [16, 64], [out, in]) uniform in
    +-sqrt(6 / fan_in) (He et al. 2015, uniform form), flattened in order, and
    the hash table [16, 2^19, 2] uniform in +-1e-4 (the hash encoding's
    initialisation). float32."""
    rng = np.random.default_rng(seed + 7000)
    parts = []
    for out_dim, in_dim in ((64, 64), (64, 64), (64, 64), (16, 64)):
        b = np.sqrt(6.0 / in_dim)
        parts.append(rng.uniform(-b, b, size=(out_dim, in_dim)))
    W = np.concatenate([p.ravel() for p in parts]).astype(np.float32)
    table = rng.uniform(-1e-4, 1e-4, size=(16, 1 << 19, 2)).astype(np.float32)
    return W, table


def surrogate_training_lights(seed: int, n: int, theta_out_deg: float = 60.0) -> np.ndarray:
    """Unit-intensity spots (I_e = 1) spread over the office ceiling for the
    surrogate's training solves: position U[0.5, 19.5] x U[0.5, 9.5] x
    U[2.5, 2.9] m, yaw U[0, 2 pi), pitch -pi/2 + U(-0.4, 0.4), theta_in
    U[25, 55] deg, theta_out fixed."""
    rng = np.random.default_rng(seed + 9000)
    rows = []
    for _ in range(n):
        pos = (rng.uniform(0.5, 19.5), rng.uniform(0.5, 9.5), rng.uniform(2.5, 2.9))
        rows.append(spot_light(pos, rng.uniform(0, 2 * np.pi), -np.pi / 2 + rng.uniform(-0.4, 0.4), 1.0,
                               np.radians(rng.uniform(25.0, 55.0)), np.radians(theta_out_deg)))
    return make_lights(rows)


def perturb_lights_in_plane(lights: np.ndarray, seed: int, pos_sigma: float = 0.3, angle_sigma: float = 0.1,
                            intensity_range=(0.7, 1.3), theta_in_deg: float = 5.0) -> np.ndarray:
    """Seeded perturbation that keeps every light at its height (ceiling
    spots stay in the room): x, y += N(0, pos_sigma), yaw, pitch +=
    N(0, angle_sigma), I_e scaled by U[intensity_range], theta_in +=
    U(-theta_in_deg, theta_in_deg) degrees (kept below theta_out)."""
    rng = np.random.default_rng(seed)
    out = np.array(lights, np.float64, copy=True)
    n = out.shape[0]
    out[:, 1:3] += rng.normal(0.0, pos_sigma, (n, 2))
    out[:, 4:6] += rng.normal(0.0, angle_sigma, (n, 2))
    out[:, 6] *= np.sqrt(rng.uniform(intensity_range[0], intensity_range[1], n))
    out[:, 7] = np.clip(out[:, 7] + np.radians(rng.uniform(-theta_in_deg, theta_in_deg, n)), 0.0, out[:, 8] - 1e-3)
    return out



# --------------------------------------------------------------------------
# Large procedural building (vectorised assembly)
# --------------------------------------------------------------------------
class _Chunks:
    """Scene arrays assembled from vectorised chunks of quads."""

    def __init__(self):
        self.xyz, self.uv, self.tile_of_tri, self.albedo, self.res, self.area = [], [], [], [], [], []
        self.n_tiles = 0

    def quads(self, p00, p10, p11, p01, pitch, albedo):
        """Quads with corners p00, p10, p11, p01 (arrays [K, 3], planar
        parallelograms), one tile each, texel counts from the texel pitch.
        Neighbouring quads must pass bitwise identical shared corners, so
        that the mesh has no cracks."""
        p00, p10, p11, p01 = (np.asarray(v, np.float64).reshape(-1, 3) for v in (p00, p10, p11, p01))
        K = p00.shape[0]
        tri = np.empty((2 * K, 3, 3))
        tri[0::2] = np.stack([p00, p10, p11], 1)
        tri[1::2] = np.stack([p00, p11, p01], 1)
        uv = np.empty((2 * K, 3, 2))
        uv[0::2] = [[0, 0], [1, 0], [1, 1]]
        uv[1::2] = [[0, 0], [1, 1], [0, 1]]
        ids = self.n_tiles + np.arange(K)
        self.xyz.append(tri)
        self.uv.append(uv)
        self.tile_of_tri.append(np.repeat(ids, 2))
        alb = np.broadcast_to(np.asarray(albedo, np.float64), (K,))
        self.albedo.append(np.repeat(alb, 2))
        a, b = p10 - p00, p01 - p00
        la, lb = np.linalg.norm(a, axis=1), np.linalg.norm(b, axis=1)
        self.res.append(np.stack([np.maximum(1, np.ceil(la / pitch - 1e-9)), np.maximum(1, np.ceil(lb / pitch - 1e-9))],
                                 1).astype(np.int32))
        self.area.append(np.linalg.norm(np.cross(a, b), axis=1))
        self.n_tiles += K

    def lattice(self, V, pitch, albedo, wrap=False):
        """Quads between neighbouring points of a vertex lattice V [nu+1, nv+1, 3]
        (with wrap, the last column closes onto the first)."""
        if wrap:
            V = np.concatenate([V, V[:1]], axis=0)
        self.quads(V[:-1, :-1].reshape(-1, 3), V[1:, :-1].reshape(-1, 3), V[1:, 1:].reshape(-1, 3),
                   V[:-1, 1:].reshape(-1, 3), pitch, albedo)

    def grid(self, corner, a, b, nu, nv, pitch, albedo):
        """A parallelogram split into nu x nv tiles on one shared lattice."""
        corner, a, b = (np.asarray(v, np.float64) for v in (corner, a, b))
        i, j = np.meshgrid(np.arange(nu + 1) / nu, np.arange(nv + 1) / nv, indexing="ij")
        self.lattice(corner + i[..., None] * a + j[..., None] * b, pitch, albedo)

    def box(self, lo, size, pitch, albedo):
        """Five faces of a box (no bottom) on its 8 corners."""
        lo = np.asarray(lo, np.float64)
        sx, sy, sz = size
        X = [lo[0], lo[0] + sx]
        Y = [lo[1], lo[1] + sy]
        Z = [lo[2], lo[2] + sz]
        P = lambda i, j, k: np.array([X[i], Y[j], Z[k]])                           # noqa: E731
        faces = [(P(0, 0, 0), P(0, 1, 0), P(0, 1, 1), P(0, 0, 1)), (P(1, 0, 0), P(1, 1, 0), P(1, 1, 1), P(1, 0, 1)),
                 (P(0, 0, 0), P(1, 0, 0), P(1, 0, 1), P(0, 0, 1)), (P(0, 1, 0), P(1, 1, 0), P(1, 1, 1), P(0, 1, 1)),
                 (P(0, 0, 1), P(1, 0, 1), P(1, 1, 1), P(0, 1, 1))]
        F = np.array(faces)
        self.quads(F[:, 0], F[:, 1], F[:, 2], F[:, 3], pitch, albedo)

    def build(self, name, **meta) -> Scene:
        return Scene(name=name,
                     xyz=np.ascontiguousarray(np.concatenate(self.xyz).astype(np.float32)),
                     uv=np.ascontiguousarray(np.concatenate(self.uv).astype(np.float32)),
                     tile=np.ascontiguousarray(np.concatenate(self.tile_of_tri).astype(np.int32)),
                     albedo=np.ascontiguousarray(np.concatenate(self.albedo).astype(np.float32)),
                     tile_res=np.ascontiguousarray(np.concatenate(self.res)),
                     tile_area=np.ascontiguousarray(np.concatenate(self.area)), meta=dict(meta))


def building(seed: int = 0, floors: int = 8, width: float = 48.0, depth: float = 24.0, storey: float = 3.5,
             slab: float = 0.3, tess: float = 0.25, pitch: float = 0.045) -> Scene:
    """A closed office building: `floors` storeys of width x depth metres,
    each a closed room between its floor (z = k storey) and the slab above
    (ceiling at z = (k + 1) storey - slab). Floors, ceilings and the four
    exterior walls are tessellated into tess x tess m tiles; per storey 21
    columns (radius 0.3 m, 32 sides x 16 rings) on a 6 m grid, 8 partitions
    (6 x 0.1 m, floor to ceiling) along the middle, and one desk or cabinet
    (5 faces, lifted 1 cm) in each 3 x 3 m cell. Albedo U[0.3, 0.8] per
    storey surface group and per box; texels at `pitch` metres."""
    rng = np.random.default_rng(seed + 11000)
    S = _Chunks()
    h = storey - slab
    nu, nv, nh = int(round(width / tess)), int(round(depth / tess)), int(np.ceil(h / tess))
    for k in range(floors):
        z0, z1 = k * storey, k * storey + h
        alb = rng.uniform(0.3, 0.8, 6)
        S.grid([0, 0, z0], [width, 0, 0], [0, depth, 0], nu, nv, pitch, alb[0])          # floor
        S.grid([0, 0, z1], [width, 0, 0], [0, depth, 0], nu, nv, pitch, alb[1])          # ceiling
        S.grid([0, 0, z0], [width, 0, 0], [0, 0, h], nu, nh, pitch, alb[2])              # walls
        S.grid([0, depth, z0], [width, 0, 0], [0, 0, h], nu, nh, pitch, alb[2])
        S.grid([0, 0, z0], [0, depth, 0], [0, 0, h], nv, nh, pitch, alb[3])
        S.grid([width, 0, z0], [0, depth, 0], [0, 0, h], nv, nh, pitch, alb[3])
        # columns: cylinders between floor and ceiling
        sides, rings, rad = 32, 16, 0.3
        phi = 2 * np.pi * np.arange(sides) / sides
        zz = z0 + h * np.arange(rings + 1) / rings
        zz[-1] = z1
        cx, cy = np.meshgrid(6.0 * np.arange(1, int(width // 6)), 6.0 * np.arange(1, int(depth // 6)), indexing="ij")
        for x, y in zip(cx.ravel(), cy.ravel()):
            V = np.stack(np.broadcast_arrays((x + rad * np.cos(phi))[:, None], (y + rad * np.sin(phi))[:, None],
                                             zz[None, :]), -1)
            S.lattice(V, pitch, alb[4], wrap=True)
        # partitions along y = depth / 2, between the columns (closed side
        # walls on one lattice around the 0.1 m thick slab)
        for i in range(int(width // 6)):
            x0, x1 = 6.0 * i + 0.5, 6.0 * i + 5.5
            y0, y1 = depth / 2 - 0.05, depth / 2 + 0.05
            n_len = int(round((x1 - x0) / tess))
            ring = np.concatenate([np.stack([x0 + (x1 - x0) * np.arange(n_len) / n_len, np.full(n_len, y0)], 1),
                                   [[x1, y0]],
                                   np.stack([x1 - (x1 - x0) * np.arange(n_len) / n_len, np.full(n_len, y1)], 1),
                                   [[x0, y1]]])
            zp = z0 + h * np.arange(nh + 1) / nh
            zp[-1] = z1
            V = np.stack(np.broadcast_arrays(ring[:, 0:1], ring[:, 1:2], zp[None, :]), -1)
            S.lattice(V, pitch, alb[5], wrap=True)
        # furniture: one box per 3 x 3 m cell
        for i in range(int(width // 3)):
            for j in range(int(depth // 3)):
                if rng.uniform() < 0.6:
                    sx, sy, sz = 1.6, 0.8, 0.75
                else:
                    sx, sy, sz = 0.8, 0.45, float(rng.uniform(1.0, 2.0))
                if rng.uniform() < 0.5:
                    sx, sy = sy, sx
                cxm = 1.5 + 3 * i + rng.uniform(-0.3, 0.3)
                cym = 1.5 + 3 * j + rng.uniform(-0.3, 0.3)
                S.box([cxm - sx / 2, cym - sy / 2, z0 + 0.01], (sx, sy, sz), pitch, float(rng.uniform(0.3, 0.8)))
    return S.build("building", seed=seed, floors=floors, pitch=pitch, tess=tess)


def building_lights(floors: int = 8, width: float = 48.0, depth: float = 24.0, storey: float = 3.5,
                    slab: float = 0.3, power: float = 200.0, size=(1.2, 0.6)) -> np.ndarray:
    """8 ceiling panels per storey (64 for 8 storeys): rectangular area
    lights 2 cm below each ceiling, facing down, at x = 9 + 12 i, y = 4.5 or
    depth - 4.5 (clear of columns and partitions)."""
    rows = []
    for k in range(floors):
        z = k * storey + storey - slab - 0.02
        for y in (4.5, depth - 4.5):
            for i in range(4):
                rows.append(area_light((9.0 + 12.0 * i, y, z), 0.0, -np.pi / 2, power, size[0], size[1]))
    return make_lights(rows)


def random_lights(n: int, seed: int, lo=(0.1, 0.1, 0.1), hi=(0.9, 0.9, 0.9)) -> np.ndarray:
    """n luminaires cycling point, spot and area, positions uniform in the box
    [lo, hi], random axes, intensity / power U[0.2, 2], spot cones
    0 <= theta_in < theta_out <= 1.4, area sizes U[0.02, 0.2] m."""
    rng = np.random.default_rng(seed + 13000)
    rows = []
    for i in range(n):
        pos = tuple(rng.uniform(lo, hi))
        yaw, pitch, I = float(rng.uniform(0, 2 * np.pi)), float(rng.uniform(-1.5, 1.5)), float(rng.uniform(0.2, 2.0))
        kind = i % 3
        if kind == 0:
            rows.append(point_light(pos, I))
        elif kind == 1:
            to = float(rng.uniform(0.2, 1.4))
            rows.append(spot_light(pos, yaw, pitch, I, float(rng.uniform(0.0, 0.95)) * to, to))
        else:
            rows.append(area_light(pos, yaw, pitch, I, float(rng.uniform(0.02, 0.2)), float(rng.uniform(0.02, 0.2))))
    return make_lights(rows)
