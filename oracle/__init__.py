"""CPU oracle for view-independent adjoint light tracing (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline and reference legs may import this package. The product path
never does.

The light transport lives in ``oracle.c`` (plain C, double precision; see its
header for what it follows in the paper). This module compiles it, loads it
with ctypes, and adds the discrete objective of Eq. 6, which is a plain numpy
sum.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def compile_source(src: str, out: str) -> None:
    """Compile one C source of the oracle into the shared library `out`
    (gcc, OpenMP, no floating-point contraction)."""
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-Wall", "-Wno-unknown-pragmas", src, "-o", out, "-lm"]
    subprocess.run(cmd, check=True)


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_lib/liboracle.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    compile_source(_SRC, tmp)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_SO)
            _declare(_lib)
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _declare(lib):
    vp, i32, i64, u32, u64, f64, ci = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                       ctypes.c_uint64, ctypes.c_double, ctypes.c_int)
    scene = [vp, vp, vp, vp, i32, vp, vp, i32]
    lib.or_forward.argtypes = scene + [vp, i32, u64, u32, u64, u64, u64, i32, vp, vp, vp, ci]
    lib.or_adjoint.argtypes = scene + [vp, i32, u64, u32, u64, u64, u64, i32, vp, vp, vp, ci]
    lib.or_paths.argtypes = scene + [vp, i32, u64, u32, u64, u64, u64, i32, vp, vp, vp, vp, vp, ci]
    lib.or_closest_hits.argtypes = [vp, i32, vp, vp, vp, i64, i32, vp, vp, vp]
    lib.or_philox4x32_10.argtypes = [vp, vp, vp]
    lib.or_philox4x32_10.restype = None
    lib.or_dflux.argtypes = [vp, u64, vp, vp, f64, f64, f64, vp, vp]
    lib.or_emit.argtypes = [vp, u64, u64, u32, u64, vp, vp, vp, vp]
    lib.or_cosine_dir.argtypes = [vp, f64, f64, vp]
    for name in ("or_forward", "or_adjoint", "or_paths", "or_closest_hits", "or_dflux", "or_emit",
                 "or_cosine_dir"):
        getattr(lib, name).restype = ctypes.c_int


def _scene_args(scene):
    arrs = (np.ascontiguousarray(scene.xyz, np.float32), np.ascontiguousarray(scene.uv, np.float32),
            np.ascontiguousarray(scene.tile, np.int32), np.ascontiguousarray(scene.albedo, np.float32),
            np.ascontiguousarray(scene.tile_res, np.int32), np.ascontiguousarray(scene.tile_area, np.float64))
    args = [_p(arrs[0]), _p(arrs[1]), _p(arrs[2]), _p(arrs[3]), scene.n_tri, _p(arrs[4]), _p(arrs[5]),
            scene.n_tiles]
    return args, arrs


def texel_areas(scene) -> np.ndarray:
    """A_t = tile area / (res_u res_v) for every texel (box basis, Eq. S.6)."""
    counts = scene.tile_res[:, 0].astype(np.int64) * scene.tile_res[:, 1]
    per = scene.tile_area / counts
    return np.repeat(per, counts).astype(np.float64)


def forward(scene, lights, seed: int, n_photons: int, max_hits: int, begin: int = 0, end: int | None = None,
            design: int = 0, threads: int = 0, counts: bool = False):
    """Alg. 1 over photons [begin, end) of an n_photons budget.

    Returns dict(E=float64[T] irradiance, count=int64[T] deposits or None,
    segments=int, deposits=int)."""
    lib = _load()
    end = n_photons if end is None else end
    sargs, keep = _scene_args(scene)
    lp = np.ascontiguousarray(lights, np.float64)
    E = np.zeros(scene.n_texels, np.float64)
    cnt = np.zeros(scene.n_texels, np.int64) if counts else None
    stats = np.zeros(2, np.float64)
    rc = lib.or_forward(*sargs, _p(lp), lp.shape[0], seed, design, n_photons, begin, end, max_hits, _p(E),
                        _p(cnt) if counts else None, _p(stats), threads)
    if rc != 0:
        raise ValueError(f"or_forward failed ({rc})")
    return dict(E=E, count=cnt, segments=int(stats[0]), deposits=int(stats[1]))


def adjoint(scene, lights, seed: int, n_photons: int, max_hits: int, w, begin: int = 0, end: int | None = None,
            design: int = 0, threads: int = 0):
    """Alg. 2 over photons [begin, end): returns (dO/dp float64[L, 8], segments).

    w[t] = alpha_t (E_t - E*_t) is dO/dPhi for a deposit into texel t."""
    lib = _load()
    end = n_photons if end is None else end
    sargs, keep = _scene_args(scene)
    lp = np.ascontiguousarray(lights, np.float64)
    wv = np.ascontiguousarray(w, np.float64)
    assert wv.shape == (scene.n_texels,)
    grad = np.zeros((lp.shape[0], 8), np.float64)
    stats = np.zeros(2, np.float64)
    rc = lib.or_adjoint(*sargs, _p(lp), lp.shape[0], seed, design, n_photons, begin, end, max_hits, _p(wv),
                        _p(grad), _p(stats), threads)
    if rc != 0:
        raise ValueError(f"or_adjoint failed ({rc})")
    return grad, int(stats[0])


def paths(scene, lights, seed: int, n_photons: int, max_hits: int, begin: int, count: int, design: int = 0,
          threads: int = 0, w=None, flux: bool = False):
    """Triangle and texel of every hit of photons [begin, begin + count); with
    adjoint weights w, also each photon's gradient term [count, 8]; with
    flux=True, also the flux Phi_i deposited at every hit [count, max_hits]
    (last in the returned tuple)."""
    lib = _load()
    sargs, keep = _scene_args(scene)
    lp = np.ascontiguousarray(lights, np.float64)
    tri = np.empty((count, max_hits), np.int32)
    tex = np.empty((count, max_hits), np.int64)
    phi = np.empty((count, max_hits), np.float64) if flux else None
    wv = np.ascontiguousarray(w, np.float64) if w is not None else None
    g = np.empty((count, 8), np.float64) if w is not None else None
    rc = lib.or_paths(*sargs, _p(lp), lp.shape[0], seed, design, n_photons, begin, count, max_hits, _p(tri),
                      _p(tex), _p(phi) if flux else None, _p(wv) if w is not None else None,
                      _p(g) if w is not None else None, threads)
    if rc != 0:
        raise ValueError(f"or_paths failed ({rc})")
    out = (tri, tex) + ((g,) if w is not None else ()) + ((phi,) if flux else ())
    return out


def loss(scene, E, target, alpha):
    """Eq. 6 for order 0 and a box basis: O = 1/2 sum_t A_t alpha_t (E_t - E*_t)^2.

    Returns (O, w) with w_t = alpha_t (E_t - E*_t) = (dO/dE_t) / A_t."""
    A = texel_areas(scene)
    r = np.asarray(E, np.float64) - np.asarray(target, np.float64)
    a = np.asarray(alpha, np.float64)
    O = 0.5 * float(np.sum(A * a * r * r))
    return O, a * r


def closest_hits(scene, o, d, skip_tile: int = -1):
    lib = _load()
    o = np.ascontiguousarray(o, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    n = o.shape[0]
    xyz = np.ascontiguousarray(scene.xyz, np.float32)
    tile = np.ascontiguousarray(scene.tile, np.int32)
    tri = np.empty(n, np.int32)
    t = np.empty(n, np.float32)
    b = np.empty((n, 3), np.float32)
    lib.or_closest_hits(_p(xyz), scene.n_tri, _p(tile), _p(o), _p(d), n, skip_tile, _p(tri), _p(t), _p(b))
    return tri, t, b


def philox(ctr, key):
    lib = _load()
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.empty(4, np.uint32)
    lib.or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def dflux(light_row, n_rays: int, x1, n1, a_emit: float = 1.0, u3: float = 0.5, u4: float = 0.5):
    """(Phi_r, dPhi_r/dp[8]) for one light with its first hit held at x1.
    For an area light the ray origin is given by the position uniforms (u3,
    u4) and a_emit is the cosine towards x1 (computed)."""
    lib = _load()
    lp = np.ascontiguousarray(light_row, np.float64).reshape(9)
    x = np.ascontiguousarray(x1, np.float64)
    n = np.ascontiguousarray(n1, np.float64)
    phi = np.zeros(1)
    out = np.zeros(8)
    lib.or_dflux(_p(lp), n_rays, _p(x), _p(n), a_emit, u3, u4, _p(phi), _p(out))
    return float(phi[0]), out


def emit(light_row, n_rays: int, seed: int, photon: int, design: int = 0, origin: bool = False):
    """Emitted direction, flux and falloff (and with origin=True the ray
    origin) of one photon of a single light."""
    lib = _load()
    lp = np.ascontiguousarray(light_row, np.float64).reshape(9)
    w = np.zeros(3)
    phi = np.zeros(1)
    a = np.zeros(1)
    x0 = np.zeros(3)
    lib.or_emit(_p(lp), n_rays, seed, design, photon, _p(w), _p(phi), _p(a), _p(x0))
    if origin:
        return w, float(phi[0]), float(a[0]), x0
    return w, float(phi[0]), float(a[0])


def cosine_dir(n, u1: float, u2: float):
    lib = _load()
    nv = np.ascontiguousarray(n, np.float64)
    w = np.zeros(3)
    lib.or_cosine_dir(_p(nv), u1, u2, _p(w))
    return w
