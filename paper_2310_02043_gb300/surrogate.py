"""Python binding of the irradiance surrogate (include/sg.h), argument
marshalling only: encoding, network, training step, and the design objective
all run in the library's CUDA kernels.

The surrogate predicts K(t, l), the irradiance a unit-intensity spot puts on
texel t, so that a design's irradiance is E_t = sum_l I_l K(t, l). It is
trained on the tracer's own per-light irradiance (``generate_solves``) and
used as a cheap first stage of the lighting optimisation (``warm_start``),
after which the tracer refines and judges the result.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lighttrace as ltr
from .lighttrace import LtError, _ptr, lights_to_struct, load_library

LEVELS = 16
TABLE_PER_LEVEL = 1 << 19
TABLE_FLOATS = LEVELS * TABLE_PER_LEVEL * 2
WEIGHTS = 3 * 64 * 64 + 16 * 64
N_IN, N_OUT = 64, 16
MAX_BATCH = 1 << 20

EXPORTED = ("sg_create", "sg_destroy", "sg_last_error", "sg_set_texels", "sg_set_params", "sg_get_params",
            "sg_set_training_data", "sg_train_step", "sg_get_gradients", "sg_response", "sg_design", "sg_network",
            "sg_encode", "sg_set_kernels")

_declared = False


def _lib():
    global _declared
    lib = load_library()
    if not _declared:
        vp, i32, i64, u64, ci, f32 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int,
                                      ctypes.c_float)
        sig = {
            "sg_create": [ctypes.POINTER(ctypes.c_void_p), ci, vp],
            "sg_destroy": [vp],
            "sg_set_texels": [vp, vp, vp, vp, i64, vp, f32],
            "sg_set_params": [vp, vp, vp, ci],
            "sg_get_params": [vp, vp, vp, ci],
            "sg_set_training_data": [vp, vp, i32, vp],
            "sg_train_step": [vp, u64, i32, f32, vp, vp],
            "sg_get_gradients": [vp, vp, vp, ci],
            "sg_response": [vp, vp, vp, ci],
            "sg_design": [vp, vp, i32, vp, vp, vp, vp, vp],
            "sg_network": [vp, vp, i32, vp, vp, vp, vp],
            "sg_encode": [vp, vp, i32, vp],
            "sg_set_kernels": [vp, ci],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib.sg_last_error.argtypes = [vp]
        lib.sg_last_error.restype = ctypes.c_char_p
        _declared = True
    return lib


class Surrogate:
    """One surrogate context on one CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = _lib()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        h = ctypes.c_void_p()
        rc = self.lib.sg_create(ctypes.byref(h), device, ctypes.c_void_p(stream))
        if rc != ltr.LT_OK:
            raise LtError(rc, "sg_create failed")
        self.h = h
        self.device = device
        self.n_texels = 0

    def close(self):
        if self.h:
            self.lib.sg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != ltr.LT_OK:
            raise LtError(rc, self.lib.sg_last_error(self.h).decode())

    def set_texels(self, pos, normal, area, lo, ext: float):
        pos = np.ascontiguousarray(pos, np.float32)
        normal = np.ascontiguousarray(normal, np.float32)
        area = np.ascontiguousarray(area, np.float32)
        lo = np.ascontiguousarray(lo, np.float32)
        self._check(self.lib.sg_set_texels(self.h, _ptr(pos)[0], _ptr(normal)[0], _ptr(area)[0], pos.shape[0],
                                           _ptr(lo)[0], float(ext)))
        self.n_texels = pos.shape[0]

    def set_params(self, weights, table):
        w, dev = _ptr(weights)
        t, dev2 = _ptr(table)
        assert dev == dev2
        self._check(self.lib.sg_set_params(self.h, w, t, dev))

    def params(self):
        W = np.empty(WEIGHTS, np.float32)
        T = np.empty((LEVELS, TABLE_PER_LEVEL, 2), np.float32)
        self._check(self.lib.sg_get_params(self.h, _ptr(W)[0], _ptr(T)[0], 0))
        return W, T

    def set_training_data(self, lights, E_obs):
        """lights [S, 9] unit-intensity spots; E_obs a CUDA tensor [S, T]."""
        self._E_obs = E_obs            # the library keeps the pointer
        arr = lights_to_struct(lights)
        ptr, dev = _ptr(E_obs)
        assert dev == 1, "E_obs must be a device tensor"
        self._check(self.lib.sg_set_training_data(self.h, arr, len(arr), ptr))

    def train_step(self, seed: int, batch: int, lr: float, samples=None) -> float:
        loss = ctypes.c_double()
        sp = None
        if samples is not None:
            samples = np.ascontiguousarray(samples, np.int32)
            assert samples.shape == (batch, 2)
            sp = _ptr(samples)[0]
        self._check(self.lib.sg_train_step(self.h, seed, batch, float(lr), sp, ctypes.byref(loss)))
        return loss.value

    def gradients(self):
        dW = np.empty(WEIGHTS, np.float32)
        dT = np.empty((LEVELS, TABLE_PER_LEVEL, 2), np.float32)
        self._check(self.lib.sg_get_gradients(self.h, _ptr(dW)[0], _ptr(dT)[0], 0))
        return dW, dT

    def response(self, light, out=None):
        """K(t, light) for every texel (host array, or into a CUDA tensor)."""
        arr = lights_to_struct(np.asarray(light, np.float64).reshape(1, 9))
        if out is None:
            out = np.empty(self.n_texels, np.float32)
        ptr, dev = _ptr(out)
        self._check(self.lib.sg_response(self.h, arr, ptr, dev))
        return out

    def design(self, lights, E_target, alpha=None, E_out=None):
        """(objective, gradient [L, 8]) of a design against a CUDA target."""
        arr = lights_to_struct(lights)
        loss = ctypes.c_double()
        grad = np.empty((len(arr), 8), np.float64)
        self._check(self.lib.sg_design(self.h, arr, len(arr), _ptr(E_target)[0],
                                       _ptr(alpha)[0] if alpha is not None else None, ctypes.byref(loss),
                                       _ptr(grad)[0], _ptr(E_out)[0] if E_out is not None else None))
        return loss.value, grad

    def network(self, X, dO=None):
        """The network on input rows X [B, 64]: returns O [B, 16], and with dO
        also dX [B, 64] and the weight gradient [WEIGHTS]."""
        X = np.ascontiguousarray(X, np.float32)
        B = X.shape[0]
        O = np.empty((B, N_OUT), np.float32)
        if dO is None:
            self._check(self.lib.sg_network(self.h, _ptr(X)[0], B, None, _ptr(O)[0], None, None))
            return O
        dO = np.ascontiguousarray(dO, np.float32)
        dX = np.empty((B, N_IN), np.float32)
        dW = np.empty(WEIGHTS, np.float32)
        self._check(self.lib.sg_network(self.h, _ptr(X)[0], B, _ptr(dO)[0], _ptr(O)[0], _ptr(dX)[0], _ptr(dW)[0]))
        return O, dX, dW

    def set_kernels(self, tcgen05: bool = True, train_tcgen05: bool = False):
        """Design objective on tcgen05 (default) or warp-level mma.sync;
        training network on mma.sync (default, measured faster) or tcgen05."""
        flags = (1 if tcgen05 else 0) | (2 if train_tcgen05 else 0)
        self._check(self.lib.sg_set_kernels(self.h, flags))

    def encode(self, xn):
        xn = np.ascontiguousarray(xn, np.float32)
        out = np.empty((xn.shape[0], 32), np.float32)
        self._check(self.lib.sg_encode(self.h, _ptr(xn)[0], xn.shape[0], _ptr(out)[0]))
        return out


def split_weights(W):
    """Flat weights -> the four matrices [out, in]."""
    W = np.asarray(W)
    return [W[0:4096].reshape(64, 64), W[4096:8192].reshape(64, 64), W[8192:12288].reshape(64, 64),
            W[12288:13312].reshape(16, 64)]
