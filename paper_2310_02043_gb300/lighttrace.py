"""Python binding of the C ABI in include/lt.h (argument marshalling only).

Every step of the light-tracing path runs in the CUDA library
``_lib/libltrace.so``; this module converts numpy arrays / torch tensors to
pointers and raises on error statuses. There is no fallback: if the library
is missing, importing works but creating a ``Tracer`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libltrace.so")

LT_OK, LT_ERR_ARG, LT_ERR_CUDA, LT_ERR_OOM, LT_ERR_STATE, LT_ERR_TIMEOUT, LT_ERR_OVERFLOW, LT_ERR_DEVICE = (
    0, -1, -2, -3, -4, -5, -6, -7)
STATUS_NAMES = {0: "LT_OK", -1: "LT_ERR_ARG", -2: "LT_ERR_CUDA", -3: "LT_ERR_OOM", -4: "LT_ERR_STATE",
                -5: "LT_ERR_TIMEOUT", -6: "LT_ERR_OVERFLOW", -7: "LT_ERR_DEVICE"}
MAX_LIGHTS = 1024
GRAD_N = 8
GRAD_FRACTION_BITS = 64   # fixed-point gradient sums count units of 2^-64 / G

# Every symbol the header declares (checked by the test suite).
EXPORTED = ("lt_version", "lt_create", "lt_destroy", "lt_set_stream", "lt_last_error", "lt_upload_scene",
            "lt_set_target", "lt_set_lights", "lt_trace_forward", "lt_texel_accumulator", "lt_get_texel_sums", "lt_loss",
            "lt_get_irradiance", "lt_texel_areas", "lt_set_adjoint_weights", "lt_trace_adjoint", "lt_debug_paths",
            "lt_get_stats", "lt_set_launch", "lt_count_work", "lt_loss_static", "lt_set_design", "lt_batch_setup",
            "lt_batch_set_lights", "lt_batch_step", "lt_batch_texel_sums", "lt_batch_irradiance",
            "lt_batch_stream", "lt_texel_centres", "lt_build_bvh", "lt_set_step_limit",
            "lt_probe_l2_read", "lt_gradient_fixed", "lt_set_tri_staging", "lt_compress_bvh")


class LtError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class lt_light(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("pos", ctypes.c_float * 3), ("yaw", ctypes.c_float),
                ("pitch", ctypes.c_float), ("p_int", ctypes.c_float), ("theta_in", ctypes.c_float),
                ("theta_out", ctypes.c_float)]


class lt_stats(ctypes.Structure):
    _fields_ = [("segments_forward", ctypes.c_uint64), ("segments_adjoint", ctypes.c_uint64),
                ("photons_forward", ctypes.c_uint64), ("photons_adjoint", ctypes.c_uint64),
                ("n_texels", ctypes.c_int64), ("n_triangles", ctypes.c_int32), ("n_nodes", ctypes.c_int32),
                ("bvh_depth", ctypes.c_int32), ("staged_nodes", ctypes.c_int32),
                ("fixed_point_scale", ctypes.c_double), ("grid_blocks", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("staged_triangles", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class lt_bvh_node(ctypes.Structure):
    _fields_ = [("lo_x", ctypes.c_float * 8), ("hi_x", ctypes.c_float * 8), ("lo_y", ctypes.c_float * 8),
                ("hi_y", ctypes.c_float * 8), ("lo_z", ctypes.c_float * 8), ("hi_z", ctypes.c_float * 8),
                ("child", ctypes.c_int32 * 8), ("inner_mask", ctypes.c_uint32), ("pad", ctypes.c_uint32 * 3)]


BVH_NODE_DTYPE = np.dtype([("lo_x", "<f4", 8), ("hi_x", "<f4", 8), ("lo_y", "<f4", 8), ("hi_y", "<f4", 8),
                           ("lo_z", "<f4", 8), ("hi_z", "<f4", 8), ("child", "<i4", 8), ("inner_mask", "<u4"),
                           ("pad", "<u4", 3)])


class lt_bvh_cnode(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("meta", ctypes.c_uint32), ("q", (ctypes.c_uint8 * 16) * 3),
                ("child", ctypes.c_int32 * 8)]


CBVH_NODE_DTYPE = np.dtype([("origin", "<f4", 3), ("meta", "<u4"), ("q", "u1", (3, 16)), ("child", "<i4", 8)])


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load libltrace.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA light-tracing library not built: {path} is missing "
                                   "(run __graft_entry__.build())")
            lib = ctypes.CDLL(path)
            _declare(lib)
            _lib = lib
    return _lib


def _declare(lib):
    vp, i32, i64, u64, ci = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
    sig = {
        "lt_version": [],
        "lt_create": [ctypes.POINTER(vp), ci, vp],
        "lt_destroy": [vp],
        "lt_set_stream": [vp, vp],
        "lt_upload_scene": [vp, vp, vp, vp, vp, i32, vp, vp, i32, ctypes.POINTER(i64)],
        "lt_set_target": [vp, vp, vp, ci],
        "lt_set_lights": [vp, vp, i32],
        "lt_trace_forward": [vp, u64, u64, i32, u64, u64],
        "lt_texel_accumulator": [vp, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_double)],
        "lt_get_texel_sums": [vp, vp, ci],
        "lt_loss": [vp, vp, ci],
        "lt_get_irradiance": [vp, vp, ci],
        "lt_texel_areas": [vp, vp, ci],
        "lt_set_adjoint_weights": [vp, vp, ci],
        "lt_trace_adjoint": [vp, u64, u64, i32, u64, u64, vp, ci],
        "lt_debug_paths": [vp, u64, u64, i32, u64, u64, vp, vp, vp],
        "lt_get_stats": [vp, ctypes.POINTER(lt_stats)],
        "lt_set_launch": [vp, i32, i32, i32],
        "lt_set_tri_staging": [vp, i32],
        "lt_compress_bvh": [vp, i32, vp],
        "lt_count_work": [vp, u64, u64, i32, u64, u64, vp],
        "lt_loss_static": [ci, vp, vp, ctypes.c_double, vp, vp, vp, i64, vp, vp, vp],
        "lt_set_design": [vp, ctypes.c_uint32],
        "lt_batch_setup": [vp, i32, vp, u64, i32],
        "lt_batch_set_lights": [vp, vp],
        "lt_batch_step": [vp, u64, u64, vp, vp, ci],
        "lt_batch_texel_sums": [vp, i32, vp, ci],
        "lt_batch_irradiance": [vp, i32, vp, ci],
        "lt_batch_stream": [vp, ctypes.POINTER(ctypes.c_void_p)],
        "lt_texel_centres": [vp, vp, vp],
        "lt_build_bvh": [vp, i32, vp, i32, vp, ctypes.POINTER(i32), ctypes.POINTER(i32)],
        "lt_set_step_limit": [vp, i32],
        "lt_probe_l2_read": [ci, u64, i32, ctypes.POINTER(ctypes.c_double)],
        "lt_gradient_fixed": [vp, vp, ctypes.POINTER(ctypes.c_double)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.lt_last_error.argtypes = [vp]
    lib.lt_last_error.restype = ctypes.c_char_p


def _ptr(x):
    """Pointer and is_device flag of a numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data_as(ctypes.c_void_p), 0
    import torch
    if isinstance(x, torch.Tensor):
        assert x.is_contiguous()
        return ctypes.c_void_p(x.data_ptr()), (1 if x.is_cuda else 0)
    raise TypeError(f"unsupported buffer type {type(x)}")


def lights_to_struct(lights: np.ndarray):
    """[n, 9] rows (type, x, y, z, yaw, pitch, p_int, theta_in, theta_out) -> lt_light array."""
    arr = np.asarray(lights, np.float64).reshape(-1, 9)
    out = (lt_light * arr.shape[0])()
    for i, row in enumerate(arr):
        out[i].type = int(row[0])
        out[i].pos[0], out[i].pos[1], out[i].pos[2] = float(row[1]), float(row[2]), float(row[3])
        out[i].yaw, out[i].pitch, out[i].p_int = float(row[4]), float(row[5]), float(row[6])
        out[i].theta_in, out[i].theta_out = float(row[7]), float(row[8])
    return out


LOSS_STATIC_MAX_TEXELS = 16777216


def loss_static(device: int, stream: int, q_ptr: int, scale: float, area, E_target, w_out, loss_out, alpha=None,
                E_out=None):
    """lt_loss_static: the objective and adjoint weights without any device
    allocation (for callers that cannot allocate). All buffers are device
    tensors; q_ptr is the device address of the int64 texel sums."""
    import torch
    lib = load_library()
    n = int(area.numel())

    def need(name, t, dtype, count):
        if t is None:
            return
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()
                and t.numel() >= count):
            raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor of at least {count} elements")

    for name, t in (("area", area), ("E_target", E_target), ("w_out", w_out), ("alpha", alpha), ("E_out", E_out)):
        need(name, t, torch.float32, n)
    need("loss_out", loss_out, torch.float64, 1)
    rc = lib.lt_loss_static(device, ctypes.c_void_p(stream), ctypes.c_void_p(q_ptr), float(scale), _ptr(area)[0],
                            _ptr(E_target)[0], _ptr(alpha)[0] if alpha is not None else None, n, _ptr(w_out)[0],
                            _ptr(E_out)[0] if E_out is not None else None, _ptr(loss_out)[0])
    if rc != LT_OK:
        raise LtError(rc, "lt_loss_static failed")


def probe_l2_read(device: int = 0, nbytes: int = 32 << 20, reps: int = 64) -> float:
    """lt_probe_l2_read: L2 read bandwidth of the device in GB/s."""
    lib = load_library()
    out = ctypes.c_double()
    rc = lib.lt_probe_l2_read(device, nbytes, reps, ctypes.byref(out))
    if rc != LT_OK:
        raise LtError(rc, "lt_probe_l2_read failed")
    return out.value


def gradient_from_fixed(sums, scale: float) -> np.ndarray:
    """dO/dp from exact gradient sums ([L, 8, 2] int64: low, high word of a
    128-bit two's-complement integer, as lt_gradient_fixed returns them, or
    the exact sum of several such arrays given as Python integers [L, 8]):
    integer x 2^-64 / scale, rounded once, as the library converts them."""
    ints = fixed_to_ints(sums) if np.asarray(sums, dtype=object).ndim == 3 else np.asarray(sums, dtype=object)
    out = np.empty(ints.shape, np.float64)
    for idx in np.ndindex(ints.shape):
        out[idx] = np.ldexp(float(int(ints[idx])), -GRAD_FRACTION_BITS) / scale
    return out


def fixed_to_ints(sums) -> np.ndarray:
    """[L, 8, 2] int64 (low, high words) -> [L, 8] array of Python integers."""
    a = np.asarray(sums, np.int64)
    out = np.empty(a.shape[:-1], dtype=object)
    for idx in np.ndindex(out.shape):
        lo, hi = int(a[idx][0]) & ((1 << 64) - 1), int(a[idx][1])
        out[idx] = (hi << 64) + lo
    return out


def build_bvh(tri_xyz):
    """lt_build_bvh: the wide BVH of [n_tri, 3, 3] float triangles, built on
    the host (no device). Returns (nodes as a BVH_NODE_DTYPE array, order
    int32 [n_tri] leaf position -> triangle, depth)."""
    lib = load_library()
    xyz = np.ascontiguousarray(tri_xyz, np.float32).reshape(-1, 9)
    n_tri = xyz.shape[0]
    n_nodes, depth = ctypes.c_int32(0), ctypes.c_int32(0)
    rc = lib.lt_build_bvh(_ptr(xyz)[0], n_tri, None, 0, None, ctypes.byref(n_nodes), ctypes.byref(depth))
    if rc != LT_OK:
        raise LtError(rc, "lt_build_bvh failed")
    nodes = np.zeros(n_nodes.value, BVH_NODE_DTYPE)
    order = np.empty(n_tri, np.int32)
    rc = lib.lt_build_bvh(_ptr(xyz)[0], n_tri, nodes.ctypes.data_as(ctypes.c_void_p), n_nodes.value, _ptr(order)[0],
                          ctypes.byref(n_nodes), ctypes.byref(depth))
    if rc != LT_OK:
        raise LtError(rc, "lt_build_bvh failed")
    return nodes, order, depth.value


def compress_bvh(nodes):
    """lt_compress_bvh: the compressed nodes (CBVH_NODE_DTYPE) of a
    BVH_NODE_DTYPE array from build_bvh, as the kernels read them when the
    BVH is not staged in shared memory."""
    lib = load_library()
    nodes = np.ascontiguousarray(nodes, BVH_NODE_DTYPE)
    out = np.zeros(len(nodes), CBVH_NODE_DTYPE)
    rc = lib.lt_compress_bvh(nodes.ctypes.data_as(ctypes.c_void_p), len(nodes), out.ctypes.data_as(ctypes.c_void_p))
    if rc != LT_OK:
        raise LtError(rc, "lt_compress_bvh failed")
    return out


class Tracer:
    """One library context on one CUDA device and stream.

    Methods map one to one onto the C ABI; see include/lt.h for semantics."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load_library()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        h = ctypes.c_void_p()
        rc = self.lib.lt_create(ctypes.byref(h), device, ctypes.c_void_p(stream))
        if rc != LT_OK:
            raise LtError(rc, "lt_create failed")
        self.h = h
        self.device = device
        self.n_texels = 0
        self.n_lights = 0

    def _check(self, rc):
        if rc != LT_OK:
            msg = self.lib.lt_last_error(self.h)
            raise LtError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.lt_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self._check(self.lib.lt_set_stream(self.h, ctypes.c_void_p(stream)))

    def upload_scene(self, scene) -> int:
        xyz = np.ascontiguousarray(scene.xyz, np.float32)
        uv = np.ascontiguousarray(scene.uv, np.float32)
        tile = np.ascontiguousarray(scene.tile, np.int32)
        alb = np.ascontiguousarray(scene.albedo, np.float32)
        res = np.ascontiguousarray(scene.tile_res, np.int32)
        area = np.ascontiguousarray(scene.tile_area, np.float64)
        n = ctypes.c_int64()
        self._check(self.lib.lt_upload_scene(self.h, _ptr(xyz)[0], _ptr(uv)[0], _ptr(tile)[0], _ptr(alb)[0],
                                             xyz.shape[0], _ptr(res)[0], _ptr(area)[0], res.shape[0],
                                             ctypes.byref(n)))
        self.n_texels = int(n.value)
        return self.n_texels

    def set_target(self, E_target, alpha=None):
        e, dev = _ptr(E_target)
        a = _ptr(alpha)[0] if alpha is not None else None
        self._check(self.lib.lt_set_target(self.h, e, a, dev))

    def set_lights(self, lights):
        arr = lights_to_struct(lights)
        self._check(self.lib.lt_set_lights(self.h, arr, len(arr)))
        self.n_lights = len(arr)

    def trace_forward(self, seed: int, n_photons: int, max_hits: int, begin: int = 0, end: int | None = None):
        end = n_photons if end is None else end
        self._check(self.lib.lt_trace_forward(self.h, seed, n_photons, max_hits, begin, end))

    def texel_accumulator(self):
        """(device pointer, scale) of the int64 texel accumulator."""
        p = ctypes.c_void_p()
        s = ctypes.c_double()
        self._check(self.lib.lt_texel_accumulator(self.h, ctypes.byref(p), ctypes.byref(s)))
        return p.value, s.value

    def texel_sums(self, out=None):
        """The int64 fixed-point texel accumulator (numpy, or into `out`)."""
        if out is None:
            out = np.empty(self.n_texels, np.int64)
        p, dev = _ptr(out)
        self._check(self.lib.lt_get_texel_sums(self.h, p, dev))
        return out

    def loss(self, out=None) -> float | None:
        """Eq. 6 objective. Returns it as a float, or writes it into `out` (a
        1-element float64 device tensor) without synchronising."""
        if out is None:
            v = ctypes.c_double()
            self._check(self.lib.lt_loss(self.h, ctypes.cast(ctypes.byref(v), ctypes.c_void_p), 0))
            return v.value
        p, dev = _ptr(out)
        self._check(self.lib.lt_loss(self.h, p, dev))
        return None

    def irradiance(self, out=None):
        if out is None:
            out = np.empty(self.n_texels, np.float32)
        p, dev = _ptr(out)
        self._check(self.lib.lt_get_irradiance(self.h, p, dev))
        return out

    def texel_areas(self, out=None):
        if out is None:
            out = np.empty(self.n_texels, np.float32)
        p, dev = _ptr(out)
        self._check(self.lib.lt_texel_areas(self.h, p, dev))
        return out

    def set_adjoint_weights(self, w):
        p, dev = _ptr(w)
        self._check(self.lib.lt_set_adjoint_weights(self.h, p, dev))

    def trace_adjoint(self, seed: int, n_photons: int, max_hits: int, begin: int = 0, end: int | None = None,
                      out=None):
        """dO/dp as float64 [n_lights, 8] (numpy, or into `out`)."""
        end = n_photons if end is None else end
        if out is None:
            out = np.zeros((self.n_lights, GRAD_N), np.float64)
        p, dev = _ptr(out)
        self._check(self.lib.lt_trace_adjoint(self.h, seed, n_photons, max_hits, begin, end, p, dev))
        return out

    def gradient_fixed(self):
        """(sums [n_lights, 8, 2] int64, scale G) of the last adjoint pass:
        dO/dp = (high 2^64 + low) 2^-64 / G, summed exactly."""
        sums = np.empty((self.n_lights, GRAD_N, 2), np.int64)
        scale = ctypes.c_double()
        self._check(self.lib.lt_gradient_fixed(self.h, _ptr(sums)[0], ctypes.byref(scale)))
        return sums, scale.value

    def debug_paths(self, seed: int, n_photons: int, max_hits: int, begin: int, count: int, grads: bool = False):
        """Per-photon record: (triangle [count, hits], texel [count, hits]) and,
        with grads=True, each photon's gradient term [count, 8]."""
        tri = np.empty((count, max_hits), np.int32)
        tex = np.empty((count, max_hits), np.int64)
        g = np.empty((count, GRAD_N), np.float64) if grads else None
        self._check(self.lib.lt_debug_paths(self.h, seed, n_photons, max_hits, begin, count, _ptr(tri)[0],
                                            _ptr(tex)[0], _ptr(g)[0] if grads else None))
        return (tri, tex, g) if grads else (tri, tex)

    def stats(self) -> dict:
        s = lt_stats()
        self._check(self.lib.lt_get_stats(self.h, ctypes.byref(s)))
        return {name: getattr(s, name) for name, _ in s._fields_}

    def count_work(self, seed: int, n_photons: int, max_hits: int, begin: int = 0, end: int | None = None) -> dict:
        """Forward pass through the counting kernel: segments, node visits,
        triangle tests and photons."""
        end = n_photons if end is None else end
        out = np.zeros(4, np.uint64)
        self._check(self.lib.lt_count_work(self.h, seed, n_photons, max_hits, begin, end, _ptr(out)[0]))
        return dict(segments=int(out[0]), node_visits=int(out[1]), tri_tests=int(out[2]), photons=int(out[3]))

    def set_design(self, design: int):
        """Philox design word of the single-design passes."""
        self._check(self.lib.lt_set_design(self.h, design))

    # ---- batched designs ----
    def batch_setup(self, lights_per_design, photons_per_design: int, max_hits: int):
        counts = np.ascontiguousarray(lights_per_design, np.int32)
        self._check(self.lib.lt_batch_setup(self.h, counts.shape[0], _ptr(counts)[0], photons_per_design, max_hits))
        self.batch_counts = counts

    def batch_set_lights(self, lights):
        """Lights of every design, concatenated in design order, rows as in set_lights."""
        arr = lights_to_struct(lights)
        assert len(arr) == int(self.batch_counts.sum())
        self._check(self.lib.lt_batch_set_lights(self.h, arr))

    def batch_step(self, seed_fwd: int, seed_adj: int, use_graph: bool = False):
        """(objective per design [D], gradient per light [total lights, 8])."""
        loss = np.empty(self.batch_counts.shape[0], np.float64)
        grad = np.empty((int(self.batch_counts.sum()), GRAD_N), np.float64)
        self._check(self.lib.lt_batch_step(self.h, seed_fwd, seed_adj, _ptr(loss)[0], _ptr(grad)[0],
                                           1 if use_graph else 0))
        return loss, grad

    def texel_centres(self):
        """(pos [T, 3], normal [T, 3]) float32 of every texel centre."""
        pos = np.empty((self.n_texels, 3), np.float32)
        nrm = np.empty((self.n_texels, 3), np.float32)
        self._check(self.lib.lt_texel_centres(self.h, _ptr(pos)[0], _ptr(nrm)[0]))
        return pos, nrm

    def batch_stream(self) -> int:
        """The batch stream handle (cudaStream_t as an int; 0 before batch_setup)."""
        out = ctypes.c_void_p()
        self._check(self.lib.lt_batch_stream(self.h, ctypes.byref(out)))
        return int(out.value or 0)

    def batch_texel_sums(self, design: int):
        out = np.empty(self.n_texels, np.int64)
        self._check(self.lib.lt_batch_texel_sums(self.h, design, _ptr(out)[0], 0))
        return out

    def batch_irradiance(self, design: int):
        out = np.empty(self.n_texels, np.float32)
        self._check(self.lib.lt_batch_irradiance(self.h, design, _ptr(out)[0], 0))
        return out

    def set_launch(self, threads_per_block: int = -1, blocks_per_sm: int = -1, smem_node_bytes: int = -1):
        """Launch shape of the tracing kernels (0: the kernel's own block
        bound, 1024 staged and through L1 / as many blocks as fit / no
        staged nodes; negative: keep)."""
        self._check(self.lib.lt_set_launch(self.h, threads_per_block, blocks_per_sm, smem_node_bytes))

    def set_tri_staging(self, max_bytes: int):
        """Shared-memory budget under which the triangles are staged with
        the nodes (0: never; default 200 KiB)."""
        self._check(self.lib.lt_set_tri_staging(self.h, max_bytes))

    def set_step_limit(self, max_steps: int = 0):
        """Node visits per ray before the tracing kernels give up on it (0:
        the default); the next synchronising call reports LT_ERR_TIMEOUT."""
        self._check(self.lib.lt_set_step_limit(self.h, max_steps))
