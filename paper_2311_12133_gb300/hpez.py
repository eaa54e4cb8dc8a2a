"""Thin ctypes binding of ``libhpez.so`` (the C-ABI of ``include/hpez.h``).

Argument marshalling only: every step of compress/decompress runs in the
library's CUDA kernels.  If the library has not been built this module
raises on use; there is no CPU fallback.  PyTorch is used only to hold
device memory and to name the CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib",
                         "libhpez.so")

HPEZ_MAX_LEVELS = 16
HPEZ_HEADER_BYTES = 512
HPEZ_OK = 0
HPEZ_EB_ABS, HPEZ_EB_REL = 0, 1
HPEZ_LINEAR, HPEZ_CUBIC_NAK, HPEZ_CUBIC_NAT, HPEZ_SPLINE_GLOBAL = 0, 1, 2, 3
HPEZ_PARADIGM_1D, HPEZ_PARADIGM_MD = 0, 1


class HpezError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        msg = hpez_strerror(code) if _lib is not None else str(code)
        super().__init__(f"{what}: hpez error {code} ({msg})")
        self.code = code


class hpez_config(ctypes.Structure):
    _fields_ = [
        ("anchor_stride", ctypes.c_int32),
        ("frozen_dim", ctypes.c_int32),
        ("chunk_syms", ctypes.c_int32),
        ("blockwise", ctypes.c_int32),
        ("block_size", ctypes.c_int32),
        ("predictor", ctypes.c_int32),
        ("alpha", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("md_inv_var", ctypes.c_double * 3),
        ("interp", ctypes.c_uint8 * HPEZ_MAX_LEVELS),
        ("paradigm", ctypes.c_uint8 * HPEZ_MAX_LEVELS),
        ("same_level", ctypes.c_uint8 * HPEZ_MAX_LEVELS),
        ("order", (ctypes.c_uint8 * 3) * HPEZ_MAX_LEVELS),
        ("h_blockmap", ctypes.c_void_p),
    ]


class hpez_tune_params(ctypes.Structure):
    _fields_ = [
        ("sample_rate", ctypes.c_double),
        ("block_rate", ctypes.c_double),
        ("sub_frac", ctypes.c_double),
        ("lorenzo_coef", ctypes.c_double),
        ("block_size", ctypes.c_int32),
        ("tune_levels", ctypes.c_int32),
        ("tune_eb", ctypes.c_int32),
        ("tune_freeze", ctypes.c_int32),
        ("tune_lorenzo", ctypes.c_int32),
        ("tune_blockwise", ctypes.c_int32),
        ("allow_natural", ctypes.c_int32),
        ("allow_same_level", ctypes.c_int32),
        ("anchor_stride", ctypes.c_int32),
    ]


class hpez_tune_report(ctypes.Structure):
    _fields_ = [
        ("stats_count", ctypes.c_uint64),
        ("mse_lin", ctypes.c_uint64 * 3),
        ("mse_cub", ctypes.c_uint64 * 3),
        ("nonsmooth_dim", ctypes.c_int32),
        ("froze", ctypes.c_int32),
        ("lorenzo_better", ctypes.c_int32),
        ("n_sample_blocks", ctypes.c_uint32),
        ("bits", ctypes.c_uint64 * 2),
        ("lorenzo_bits", ctypes.c_uint64 * 2),
        ("level_choice", (ctypes.c_uint8 * HPEZ_MAX_LEVELS) * 2),
        ("level_score", (ctypes.c_uint64 * HPEZ_MAX_LEVELS) * 2),
    ]


class hpez_field_desc(ctypes.Structure):
    _fields_ = [
        ("d_in", ctypes.c_void_p),
        ("ndim", ctypes.c_int32),
        ("eb_mode", ctypes.c_int32),
        ("dims", ctypes.c_uint64 * 3),
        ("eb", ctypes.c_double),
        ("cfg", ctypes.POINTER(hpez_config)),
        ("d_out", ctypes.c_void_p),
        ("out_cap", ctypes.c_uint64),
    ]


class hpez_stream_desc(ctypes.Structure):
    _fields_ = [
        ("d_in", ctypes.c_void_p),
        ("in_size", ctypes.c_uint64),
        ("h_header", ctypes.c_void_p),
        ("d_out", ctypes.c_void_p),
        ("out_cap_elems", ctypes.c_uint64),
    ]


class hpez_level_key(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("cls", ctypes.c_int32 * 3),
                ("stride", ctypes.c_int32), ("interp", ctypes.c_int32),
                ("paradigm", ctypes.c_int32), ("decomp", ctypes.c_int32)]

    def astuple(self):
        return (self.ndim, *self.cls, self.stride, self.interp, self.paradigm, self.decomp)


class hpez_level_sched(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int32), ("tile", ctypes.c_int32 * 3),
                ("chunks", ctypes.c_int32), ("time_us", ctypes.c_float)]

    def astuple(self):
        return (self.family, *self.tile, self.chunks)


HPEZ_FAM_LEVEL3D, HPEZ_FAM_MD3W, HPEZ_FAM_MD3, HPEZ_FAM_FUSED, HPEZ_FAM_PASS = 1, 2, 3, 4, 5


class hpez_request(ctypes.Structure):
    _fields_ = [
        ("op", ctypes.c_int32),
        ("ndim", ctypes.c_int32),
        ("dims", ctypes.c_uint64 * 3),
        ("eb_mode", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("eb", ctypes.c_double),
        ("cfg", ctypes.POINTER(hpez_config)),
        ("h_in", ctypes.c_void_p),
        ("in_bytes", ctypes.c_uint64),
        ("h_out", ctypes.c_void_p),
        ("out_cap", ctypes.c_uint64),
    ]


HPEZ_REQ_COMPRESS, HPEZ_REQ_DECOMPRESS = 0, 1

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(
                f"{_LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` "
                "(there is no fallback implementation)")
        L = ctypes.CDLL(_LIB_PATH)
        vp, u64, u64p = ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)
        cfgp = ctypes.POINTER(hpez_config)
        sig = {
            "hpez_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int]),
            "hpez_destroy": (ctypes.c_int, [vp]),
            "hpez_default_config": (ctypes.c_int, [ctypes.c_int, cfgp]),
            "hpez_compress_bound": (ctypes.c_int, [ctypes.c_int, u64p, u64p]),
            "hpez_compress": (ctypes.c_int, [vp, vp, ctypes.c_int, u64p,
                                             ctypes.c_int, ctypes.c_double,
                                             cfgp, vp, u64, u64p, vp]),
            "hpez_decompress": (ctypes.c_int, [vp, vp, u64, vp, u64, vp]),
            "hpez_compress_async": (ctypes.c_int, [vp, vp, ctypes.c_int, u64p,
                                                   ctypes.c_int, ctypes.c_double,
                                                   cfgp, vp, u64, vp, vp, vp]),
            "hpez_decompress_async": (ctypes.c_int, [vp, vp, u64, vp, vp, u64, vp, vp]),
            "hpez_compress_host": (ctypes.c_int, [vp, vp, ctypes.c_int, u64p,
                                                  ctypes.c_int, ctypes.c_double,
                                                  cfgp, vp, u64, u64p, vp]),
            "hpez_decompress_host": (ctypes.c_int, [vp, vp, u64, vp, u64, vp]),
            "hpez_inspect": (ctypes.c_int, [vp, u64, ctypes.POINTER(ctypes.c_int),
                                            u64p, ctypes.POINTER(ctypes.c_double)]),
            "hpez_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "hpez_profile_enable": (ctypes.c_int, [vp, ctypes.c_int]),
            "hpez_profile_get": (ctypes.c_int, [vp, ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_double), u64p]),
            "hpez_profile_phase_name": (ctypes.c_char_p, [ctypes.c_int]),
            "hpez_launch_count": (ctypes.c_int, [vp, u64p]),
            "hpez_set_option": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int64]),
            "hpez_decompress_noalloc": (ctypes.c_int, [vp, u64, vp, u64, vp]),
            "hpez_default_tune_params": (ctypes.c_int,
                                         [ctypes.POINTER(hpez_tune_params)]),
            "hpez_blockmap_size": (u64, [ctypes.c_int, u64p, ctypes.c_int]),
            "hpez_compress_auto": (ctypes.c_int, [vp, vp, ctypes.c_int, u64p,
                                                  ctypes.c_int, ctypes.c_double,
                                                  ctypes.POINTER(hpez_tune_params),
                                                  vp, u64, u64p,
                                                  ctypes.POINTER(hpez_tune_report), vp]),
            "hpez_compress_auto_host": (ctypes.c_int, [vp, vp, ctypes.c_int, u64p,
                                                       ctypes.c_int, ctypes.c_double,
                                                       ctypes.POINTER(hpez_tune_params),
                                                       vp, u64, u64p, vp]),
            "hpez_psnr": (ctypes.c_int, [vp, vp, vp, u64, ctypes.c_double,
                                         ctypes.POINTER(ctypes.c_double), u64p, vp]),
            "hpez_compress_psnr": (ctypes.c_int, [vp, vp, ctypes.c_int, u64p, ctypes.c_double,
                                                  ctypes.POINTER(hpez_tune_params), vp, u64,
                                                  u64p, ctypes.POINTER(ctypes.c_double),
                                                  ctypes.POINTER(ctypes.c_double), vp]),
            "hpez_compress_typed": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, u64p,
                                                   ctypes.c_int, ctypes.c_double, cfgp,
                                                   ctypes.c_int,
                                                   ctypes.POINTER(hpez_tune_params), vp, u64,
                                                   u64p, vp]),
            "hpez_decompress_typed": (ctypes.c_int, [vp, vp, u64, vp, ctypes.c_int, u64, vp]),
            "hpez_lossless_encode": (ctypes.c_int, [vp, vp, u64, vp, u64, u64p, vp]),
            "hpez_lossless_decode": (ctypes.c_int, [vp, vp, u64, vp, u64, u64p, vp]),
            "hpez_tune": (ctypes.c_int, [vp, vp, ctypes.c_int, u64p, ctypes.c_int,
                                         ctypes.c_double,
                                         ctypes.POINTER(hpez_tune_params), cfgp,
                                         vp, u64, ctypes.POINTER(hpez_tune_report),
                                         vp]),
            "hpez_batch_create_compress": (ctypes.c_int, [vp, ctypes.c_int,
                                                          ctypes.POINTER(hpez_field_desc),
                                                          ctypes.POINTER(vp)]),
            "hpez_batch_create_decompress": (ctypes.c_int, [vp, ctypes.c_int,
                                                            ctypes.POINTER(hpez_stream_desc),
                                                            ctypes.POINTER(vp)]),
            "hpez_batch_run": (ctypes.c_int, [vp, vp]),
            "hpez_batch_run_graph": (ctypes.c_int, [vp, vp]),
            "hpez_batch_results": (ctypes.c_int, [vp, vp, u64p,
                                                  ctypes.POINTER(ctypes.c_int32)]),
            "hpez_batch_launch_count": (ctypes.c_int, [vp, u64p, u64p]),
            "hpez_batch_destroy": (ctypes.c_int, [vp]),
            "hpez_server_create": (ctypes.c_int, [vp, u64, ctypes.c_int, vp,
                                                  ctypes.POINTER(vp)]),
            "hpez_server_submit": (ctypes.c_int, [vp, ctypes.POINTER(hpez_request), u64p]),
            "hpez_server_step": (ctypes.c_int, [vp]),
            "hpez_server_poll": (ctypes.c_int, [vp, ctypes.c_int, u64p,
                                                ctypes.POINTER(ctypes.c_int32), u64p,
                                                ctypes.POINTER(ctypes.c_double),
                                                ctypes.POINTER(ctypes.c_int)]),
            "hpez_server_stats": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int),
                                                 ctypes.POINTER(ctypes.c_int), u64p,
                                                 u64p, u64p]),
            "hpez_server_destroy": (ctypes.c_int, [vp]),
            "hpez_tuning_create": (ctypes.c_int, [ctypes.POINTER(vp)]),
            "hpez_tuning_destroy": (ctypes.c_int, [vp]),
            "hpez_tuning_set": (ctypes.c_int, [vp, ctypes.POINTER(hpez_level_key),
                                               ctypes.POINTER(hpez_level_sched)]),
            "hpez_tuning_get": (ctypes.c_int, [vp, ctypes.POINTER(hpez_level_key),
                                               ctypes.POINTER(hpez_level_sched),
                                               ctypes.POINTER(ctypes.c_int)]),
            "hpez_tuning_count": (ctypes.c_int, [vp, u64p]),
            "hpez_tuning_save": (ctypes.c_int, [vp, ctypes.c_char_p]),
            "hpez_tuning_load": (ctypes.c_int, [vp, ctypes.c_char_p]),
            "hpez_level_key_of": (ctypes.c_int, [ctypes.c_int, u64p, cfgp, ctypes.c_int,
                                                 ctypes.c_int,
                                                 ctypes.POINTER(hpez_level_key)]),
            "hpez_use_tuning": (ctypes.c_int, [vp, vp]),
            "hpez_tuning_search": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, u64p, ctypes.c_int,
                                                  ctypes.c_double, cfgp, ctypes.c_int,
                                                  ctypes.c_int, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def exported_symbols() -> list[str]:
    """Names of the C-ABI entry points this binding expects."""
    return ["hpez_create", "hpez_destroy", "hpez_default_config",
            "hpez_compress_bound", "hpez_compress", "hpez_decompress",
            "hpez_compress_host", "hpez_decompress_host", "hpez_inspect",
            "hpez_strerror", "hpez_profile_enable", "hpez_profile_get",
            "hpez_profile_phase_name", "hpez_launch_count", "hpez_set_option",
            "hpez_decompress_noalloc", "hpez_default_tune_params",
            "hpez_blockmap_size", "hpez_tune", "hpez_compress_auto",
            "hpez_compress_auto_host", "hpez_batch_create_compress",
            "hpez_batch_create_decompress", "hpez_batch_run", "hpez_batch_run_graph",
            "hpez_batch_results", "hpez_batch_launch_count", "hpez_batch_destroy",
            "hpez_server_create", "hpez_server_submit", "hpez_server_step",
            "hpez_server_poll", "hpez_server_stats", "hpez_server_destroy",
            "hpez_psnr", "hpez_compress_psnr", "hpez_compress_typed",
            "hpez_decompress_typed", "hpez_lossless_encode", "hpez_lossless_decode",
            "hpez_tuning_create", "hpez_tuning_destroy", "hpez_tuning_set",
            "hpez_tuning_get", "hpez_tuning_count", "hpez_tuning_save",
            "hpez_tuning_load", "hpez_level_key_of", "hpez_use_tuning",
            "hpez_tuning_search", "hpez_compress_async", "hpez_decompress_async"]


def _check(rc: int, what: str):
    if rc != HPEZ_OK:
        raise HpezError(rc, what)


def _dims(shape):
    return (ctypes.c_uint64 * 3)(*([int(v) for v in shape] + [1] * (3 - len(shape))))


# --------------------------------------------------------------------------
# the C-ABI, name for name
# --------------------------------------------------------------------------
def hpez_strerror(code: int) -> str:
    return _load().hpez_strerror(code).decode()


def hpez_create(device: int = 0) -> int:
    h = ctypes.c_void_p(0)
    _check(_load().hpez_create(ctypes.byref(h), device), "hpez_create")
    return h.value


def hpez_destroy(ctx: int) -> None:
    _check(_load().hpez_destroy(ctx), "hpez_destroy")


def hpez_default_config(ndim: int) -> hpez_config:
    c = hpez_config()
    _check(_load().hpez_default_config(ndim, ctypes.byref(c)), "hpez_default_config")
    return c


def hpez_compress_bound(shape) -> int:
    out = ctypes.c_uint64(0)
    _check(_load().hpez_compress_bound(len(shape), _dims(shape), ctypes.byref(out)),
           "hpez_compress_bound")
    return out.value


def hpez_compress(ctx, d_in: int, shape, eb_mode: int, eb: float,
                  cfg: hpez_config | None, d_out: int, out_cap: int,
                  stream: int = 0) -> int:
    size = ctypes.c_uint64(0)
    _check(_load().hpez_compress(ctx, d_in, len(shape), _dims(shape), eb_mode,
                                 float(eb), ctypes.byref(cfg) if cfg is not None else None,
                                 d_out, out_cap, ctypes.byref(size), stream or None),
           "hpez_compress")
    return size.value


def hpez_decompress(ctx, d_in: int, in_size: int, d_out: int,
                    out_cap_elems: int, stream: int = 0) -> None:
    _check(_load().hpez_decompress(ctx, d_in, in_size, d_out, out_cap_elems,
                                   stream or None), "hpez_decompress")


def hpez_level_key_of(shape, cfg: hpez_config | None, level: int, decomp: bool) -> tuple:
    k = hpez_level_key()
    _check(_load().hpez_level_key_of(len(shape), _dims(shape), _cfg_ptr(cfg), level,
                                     int(bool(decomp)), ctypes.byref(k)), "hpez_level_key_of")
    return k.astuple()


def hpez_use_tuning(ctx, tuning) -> None:
    _check(_load().hpez_use_tuning(ctx, tuning.handle if tuning is not None else None),
           "hpez_use_tuning")


class Tuning:
    """A table of level schedules of the batched and served forms (host
    memory): keys are tuples (ndim, cls0, cls1, cls2, stride, interp,
    paradigm, decomp), values (family, tile0, tile1, tile2, chunks)."""

    def __init__(self, path: str | None = None):
        h = ctypes.c_void_p(0)
        _check(_load().hpez_tuning_create(ctypes.byref(h)), "hpez_tuning_create")
        self.handle = h.value
        if path is not None:
            self.load(path)

    @staticmethod
    def _key(key):
        k = hpez_level_key()
        k.ndim, k.cls[0], k.cls[1], k.cls[2], k.stride, k.interp, k.paradigm, k.decomp = key
        return k

    def set(self, key, family: int, tile=(0, 0, 0), chunks: int = 0, time_us: float = 0.0):
        v = hpez_level_sched()
        v.family = family
        v.tile[0], v.tile[1], v.tile[2] = tile
        v.chunks = chunks
        v.time_us = time_us
        _check(_load().hpez_tuning_set(self.handle, ctypes.byref(self._key(key)),
                                       ctypes.byref(v)), "hpez_tuning_set")

    def get(self, key):
        v = hpez_level_sched()
        found = ctypes.c_int(0)
        _check(_load().hpez_tuning_get(self.handle, ctypes.byref(self._key(key)),
                                       ctypes.byref(v), ctypes.byref(found)), "hpez_tuning_get")
        return v if found.value else None

    def __len__(self):
        n = ctypes.c_uint64(0)
        _check(_load().hpez_tuning_count(self.handle, ctypes.byref(n)), "hpez_tuning_count")
        return n.value

    def save(self, path: str):
        _check(_load().hpez_tuning_save(self.handle, os.fsencode(path)), "hpez_tuning_save")

    def load(self, path: str):
        _check(_load().hpez_tuning_load(self.handle, os.fsencode(path)), "hpez_tuning_load")

    def search(self, ctx, x, eb: float, eb_mode: int = 1, cfg: hpez_config | None = None,
               copies: int = 0, reps: int = 3, stream=None):
        """The offline search for the class of device field `x` (float32,
        contiguous): the fastest schedule of each level and direction."""
        _check(_load().hpez_tuning_search(ctx.handle if hasattr(ctx, "handle") else ctx,
                                          self.handle, x.data_ptr(), x.dim(), _dims(x.shape),
                                          eb_mode, float(eb), _cfg_ptr(cfg), copies, reps,
                                          Context._stream(stream)), "hpez_tuning_search")

    def close(self):
        if self.handle:
            _load().hpez_tuning_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hpez_compress_async(ctx, d_in: int, shape, eb_mode: int, eb: float,
                        cfg: hpez_config | None, d_out: int, out_cap: int, d_size: int,
                        d_status: int, stream: int = 0) -> None:
    """Enqueue a compress; the size (u64) and status (int32) land at the
    device addresses d_size / d_status."""
    _check(_load().hpez_compress_async(ctx, d_in, len(shape), _dims(shape), eb_mode, float(eb),
                                       ctypes.byref(cfg) if cfg is not None else None, d_out,
                                       out_cap, d_size, d_status, stream or None),
           "hpez_compress_async")


def hpez_decompress_async(ctx, d_in: int, in_size: int, header: bytes, d_out: int,
                          out_cap_elems: int, d_status: int, stream: int = 0) -> None:
    """Enqueue a decompress planned from `header` (the stream's first 512
    bytes); the status (int32) lands at the device address d_status."""
    hb = ctypes.create_string_buffer(bytes(header[:HPEZ_HEADER_BYTES]), HPEZ_HEADER_BYTES)
    _check(_load().hpez_decompress_async(ctx, d_in, in_size, hb, d_out, out_cap_elems,
                                         d_status, stream or None), "hpez_decompress_async")


HPEZ_NOALLOC_MAX_POINTS = 2097152
HPEZ_ERR_TOO_LARGE = -10


def hpez_decompress_noalloc(d_in: int, in_size: int, d_out: int,
                            out_cap_elems: int, stream: int = 0) -> None:
    """Decompress with no allocation at all: scratch is a fixed device array
    inside the library (fields up to HPEZ_NOALLOC_MAX_POINTS points), for
    callers that may not allocate; concurrent calls race."""
    _check(_load().hpez_decompress_noalloc(d_in, in_size, d_out, out_cap_elems,
                                           stream or None), "hpez_decompress_noalloc")


def hpez_compress_host(ctx, h_in: np.ndarray, eb_mode: int, eb: float,
                       cfg: hpez_config | None, h_out: np.ndarray,
                       stream: int = 0) -> int:
    assert h_in.dtype == np.float32 and h_in.flags.c_contiguous
    size = ctypes.c_uint64(0)
    _check(_load().hpez_compress_host(
        ctx, h_in.ctypes.data, h_in.ndim, _dims(h_in.shape), eb_mode, float(eb),
        ctypes.byref(cfg) if cfg is not None else None, h_out.ctypes.data,
        h_out.nbytes, ctypes.byref(size), stream or None), "hpez_compress_host")
    return size.value


def hpez_decompress_host(ctx, h_in: np.ndarray, in_size: int,
                         h_out: np.ndarray, stream: int = 0) -> None:
    assert h_out.dtype == np.float32 and h_out.flags.c_contiguous
    _check(_load().hpez_decompress_host(ctx, h_in.ctypes.data, in_size,
                                        h_out.ctypes.data, h_out.size,
                                        stream or None), "hpez_decompress_host")


def hpez_inspect(header: bytes):
    buf = np.frombuffer(header, dtype=np.uint8)
    nd = ctypes.c_int(0)
    dims = (ctypes.c_uint64 * 3)()
    eb = ctypes.c_double(0)
    _check(_load().hpez_inspect(buf.ctypes.data, buf.size, ctypes.byref(nd), dims,
                                ctypes.byref(eb)), "hpez_inspect")
    return nd.value, tuple(int(dims[i]) for i in range(nd.value)), eb.value


HPEZ_PH_RANGE, HPEZ_PH_ANCHORS, HPEZ_PH_HIST, HPEZ_PH_CODEBOOK = 0, 1, 2, 3
HPEZ_PH_ENCODE, HPEZ_PH_PACK, HPEZ_PH_OUTLIERS, HPEZ_PH_FINALIZE = 4, 5, 6, 7
HPEZ_PH_DEC_PREP, HPEZ_PH_DECODE, HPEZ_PH_SCATTER = 8, 9, 10
HPEZ_PH_LEVEL, HPEZ_PH_DLEVEL = 11, 27
HPEZ_PH_TUNE_STATS, HPEZ_PH_TUNE_LEVELS, HPEZ_PH_TUNE_EB = 43, 44, 45
HPEZ_PH_TUNE_LORENZO, HPEZ_PH_TUNE_BLOCKS, HPEZ_PROFILE_PHASES = 46, 47, 48


def hpez_profile_enable(ctx, enable: bool) -> None:
    _check(_load().hpez_profile_enable(ctx, 1 if enable else 0), "hpez_profile_enable")


def hpez_profile_get(ctx, phase: int):
    ms = ctypes.c_double(0)
    cnt = ctypes.c_uint64(0)
    _check(_load().hpez_profile_get(ctx, phase, ctypes.byref(ms), ctypes.byref(cnt)),
           "hpez_profile_get")
    return ms.value, cnt.value


def hpez_profile_phase_name(phase: int) -> str:
    return _load().hpez_profile_phase_name(phase).decode()


HPEZ_OPT_FUSED_LEVELS, HPEZ_OPT_TILE_E0, HPEZ_OPT_TILE_E1 = 1, 2, 3
HPEZ_OPT_TILE_E2, HPEZ_OPT_FUSED_SMEM, HPEZ_OPT_LEVEL3D = 4, 5, 6
HPEZ_OPT_STREAM_LEVELS = 7
HPEZ_OPT_DROP_COPY = 8
HPEZ_OPT_STREAM_CHUNKS, HPEZ_OPT_LORENZO_CTAS, HPEZ_OPT_WARP_LEVELS = 9, 10, 11
HPEZ_OPT_BATCH_CTAS = 12


def hpez_set_option(ctx, option: int, value: int) -> None:
    _check(_load().hpez_set_option(ctx, option, int(value)), "hpez_set_option")


def hpez_launch_count(ctx) -> int:
    n = ctypes.c_uint64(0)
    _check(_load().hpez_launch_count(ctx, ctypes.byref(n)), "hpez_launch_count")
    return n.value


def hpez_default_tune_params(**kw) -> hpez_tune_params:
    t = hpez_tune_params()
    _check(_load().hpez_default_tune_params(ctypes.byref(t)), "hpez_default_tune_params")
    for k, v in kw.items():
        setattr(t, k, v)
    return t


def hpez_compress_auto(ctx, d_in: int, shape, eb_mode: int, eb: float,
                       tp: hpez_tune_params | None, d_out: int, out_cap: int,
                       stream: int = 0, report: bool = False):
    """Tune (Sec. 6) then compress; returns the stream size (and the tuning
    report when asked)."""
    size = ctypes.c_uint64(0)
    rep = hpez_tune_report() if report else None
    _check(_load().hpez_compress_auto(ctx, d_in, len(shape), _dims(shape), eb_mode,
                                      float(eb), ctypes.byref(tp) if tp is not None else None,
                                      d_out, out_cap, ctypes.byref(size),
                                      ctypes.byref(rep) if rep is not None else None,
                                      stream or None), "hpez_compress_auto")
    return (size.value, rep) if report else size.value


HPEZ_DTYPE_F32, HPEZ_DTYPE_I16, HPEZ_DTYPE_U16, HPEZ_DTYPE_I32 = 0, 1, 2, 3


def hpez_psnr(ctx, d_x: int, d_y: int, n: int, unit: float, stream: int = 0):
    """(PSNR in dB, fixed-point squared-error sum) of y against x."""
    ps = ctypes.c_double(0)
    sse = ctypes.c_uint64(0)
    _check(_load().hpez_psnr(ctx, d_x, d_y, n, float(unit), ctypes.byref(ps),
                             ctypes.byref(sse), stream or None), "hpez_psnr")
    return ps.value, sse.value


def hpez_compress_psnr(ctx, d_in: int, shape, target_db: float,
                       tp: hpez_tune_params | None, d_out: int, out_cap: int,
                       stream: int = 0):
    """Eq. 1 with M = PSNR: (stream size, absolute bound found, its PSNR)."""
    size = ctypes.c_uint64(0)
    eb = ctypes.c_double(0)
    ps = ctypes.c_double(0)
    _check(_load().hpez_compress_psnr(ctx, d_in, len(shape), _dims(shape), float(target_db),
                                      ctypes.byref(tp) if tp is not None else None, d_out,
                                      out_cap, ctypes.byref(size), ctypes.byref(eb),
                                      ctypes.byref(ps), stream or None), "hpez_compress_psnr")
    return size.value, eb.value, ps.value


def hpez_compress_typed(ctx, d_in: int, dtype: int, shape, eb_mode: int, eb: float,
                        cfg: hpez_config | None, tune: bool, tp: hpez_tune_params | None,
                        d_out: int, out_cap: int, stream: int = 0) -> int:
    size = ctypes.c_uint64(0)
    _check(_load().hpez_compress_typed(ctx, d_in, dtype, len(shape), _dims(shape), eb_mode,
                                       float(eb), ctypes.byref(cfg) if cfg is not None else None,
                                       int(tune), ctypes.byref(tp) if tp is not None else None,
                                       d_out, out_cap, ctypes.byref(size), stream or None),
           "hpez_compress_typed")
    return size.value


def hpez_decompress_typed(ctx, d_in: int, in_size: int, d_out: int, dtype: int,
                          out_cap_elems: int, stream: int = 0) -> None:
    _check(_load().hpez_decompress_typed(ctx, d_in, in_size, d_out, dtype, out_cap_elems,
                                         stream or None), "hpez_decompress_typed")


def hpez_lossless_encode(ctx, d_in: int, in_size: int, d_out: int, out_cap: int,
                         stream: int = 0) -> int:
    """The lossless stage (Sec. 4 Step 5) over a stream; the output size."""
    size = ctypes.c_uint64(0)
    _check(_load().hpez_lossless_encode(ctx, d_in, in_size, d_out, out_cap, ctypes.byref(size),
                                        stream or None), "hpez_lossless_encode")
    return size.value


def hpez_lossless_decode(ctx, d_in: int, in_size: int, d_out: int, out_cap: int,
                         stream: int = 0) -> int:
    size = ctypes.c_uint64(0)
    _check(_load().hpez_lossless_decode(ctx, d_in, in_size, d_out, out_cap, ctypes.byref(size),
                                        stream or None), "hpez_lossless_decode")
    return size.value


def hpez_compress_auto_host(ctx, h_in: np.ndarray, eb_mode: int, eb: float,
                            tp: hpez_tune_params | None, h_out: np.ndarray,
                            stream: int = 0) -> int:
    assert h_in.dtype == np.float32 and h_in.flags.c_contiguous
    size = ctypes.c_uint64(0)
    _check(_load().hpez_compress_auto_host(
        ctx, h_in.ctypes.data, h_in.ndim, _dims(h_in.shape), eb_mode, float(eb),
        ctypes.byref(tp) if tp is not None else None, h_out.ctypes.data, h_out.nbytes,
        ctypes.byref(size), stream or None), "hpez_compress_auto_host")
    return size.value


def hpez_blockmap_size(shape, block_size: int = 32) -> int:
    return int(_load().hpez_blockmap_size(len(shape), _dims(shape), block_size))


def hpez_tune(ctx, d_in: int, shape, eb_mode: int, eb: float,
              tp: hpez_tune_params | None = None, stream: int = 0):
    """Runs the Sec. 6 tuner on a device field; returns (config, report).
    The config keeps a reference to its host block map."""
    bs = tp.block_size if tp is not None else 32
    nbm = hpez_blockmap_size(shape, bs) if bs >= 1 else 0
    bm = np.zeros(max(nbm, 1), np.uint8)
    cfg = hpez_config()
    rep = hpez_tune_report()
    _check(_load().hpez_tune(ctx, d_in, len(shape), _dims(shape), eb_mode, float(eb),
                             ctypes.byref(tp) if tp is not None else None,
                             ctypes.byref(cfg), bm.ctypes.data, bm.size,
                             ctypes.byref(rep), stream or None), "hpez_tune")
    cfg._blockmap_ref = bm[:nbm] if cfg.blockwise else None
    if cfg.blockwise:
        cfg.h_blockmap = cfg._blockmap_ref.ctypes.data
    return cfg, rep


# --------------------------------------------------------------------------
# config helper
# --------------------------------------------------------------------------
def make_config(ndim: int, *, anchor_stride=None, frozen_dim=-1, chunk_syms=16384,
                alpha=1.0, beta=1.0, md_inv_var=(1, 1, 1), interp=HPEZ_CUBIC_NAK,
                paradigm=HPEZ_PARADIGM_1D, same_level=0, order=None,
                blockmap=None, block_size=32, predictor=0) -> hpez_config:
    """Config with one setting for all levels unless per-level lists are
    given (index l-1); ``order`` may be one order or a per-level list;
    ``predictor`` 1 or 2 selects the Lorenzo predictor of that order."""
    c = hpez_default_config(ndim)
    if anchor_stride is not None:
        c.anchor_stride = anchor_stride
    c.frozen_dim = frozen_dim
    c.chunk_syms = chunk_syms
    c.alpha, c.beta = float(alpha), float(beta)
    for d in range(3):
        c.md_inv_var[d] = float(md_inv_var[d])
    dims = [d for d in range(ndim) if d != frozen_dim]
    def per(v, l):
        # per-level lists shorter than the level count repeat their last entry
        if isinstance(v, (list, tuple)):
            return v[l] if l < len(v) else v[-1]
        return v

    for l in range(HPEZ_MAX_LEVELS):
        c.interp[l] = per(interp, l)
        c.paradigm[l] = per(paradigm, l)
        c.same_level[l] = per(same_level, l)
        if order is None:
            o = dims
        elif isinstance(order[0], (list, tuple)):
            o = order[l] if l < len(order) else order[-1]
        else:
            o = order
        for j in range(3):
            c.order[l][j] = o[j] if j < len(o) else 255
    c.block_size = block_size
    c.blockwise = 0
    c.predictor = predictor
    c._blockmap_ref = None
    if blockmap is not None:
        bm = np.ascontiguousarray(blockmap, dtype=np.uint8)
        c._blockmap_ref = bm
        c.h_blockmap = bm.ctypes.data
        c.blockwise = 1
    return c


# --------------------------------------------------------------------------
# torch convenience layer (device memory + streams only)
# --------------------------------------------------------------------------
class Context:
    """Owns one hpez_ctx on a CUDA device."""

    def __init__(self, device: int = 0):
        import weakref
        self.device = device
        self.handle = hpez_create(device)
        # batches and servers planned on this context: destroyed before it
        self._children = weakref.WeakSet()

    def close(self):
        if self.handle:
            for c in list(self._children):
                c.close()
            hpez_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _stream(stream):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        return stream.cuda_stream

    def compress(self, x, eb: float, eb_mode: int = HPEZ_EB_REL,
                 config: hpez_config | None = None, out=None, stream=None):
        """x: contiguous float32 CUDA tensor.  Returns (uint8 tensor, size)."""
        import torch
        assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
        cap = hpez_compress_bound(tuple(x.shape))
        if out is None or out.numel() < cap:
            out = torch.empty(cap, dtype=torch.uint8, device=x.device)
        size = hpez_compress(self.handle, x.data_ptr(), tuple(x.shape), eb_mode, eb,
                             config, out.data_ptr(), out.numel(), self._stream(stream))
        return out, size

    def tune(self, x, eb: float, eb_mode: int = HPEZ_EB_REL,
             params: hpez_tune_params | None = None, stream=None):
        """x: contiguous float32 CUDA tensor.  Returns (config, report)."""
        import torch
        assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
        return hpez_tune(self.handle, x.data_ptr(), tuple(x.shape), eb_mode, eb,
                         params, self._stream(stream))

    def decompress(self, stream_buf, size: int, out=None, shape=None, stream=None):
        """stream_buf: uint8 CUDA tensor holding `size` bytes."""
        import torch
        if shape is None:
            hdr = stream_buf[:HPEZ_HEADER_BYTES].cpu().numpy().tobytes()
            _, shape, _ = hpez_inspect(hdr)
        n = int(np.prod(shape))
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=stream_buf.device)
        hpez_decompress(self.handle, stream_buf.data_ptr(), size, out.data_ptr(), n,
                        self._stream(stream))
        return out


# --------------------------------------------------------------------------
# batched and served forms
# --------------------------------------------------------------------------
def _cfg_ptr(cfg):
    return ctypes.pointer(cfg) if cfg is not None else None


class Batch:
    """A batch of compress (or decompress) requests bound to device buffers.

    compress: ``fields`` = list of (x tensor, eb, eb_mode, config or None);
    output buffers are allocated here (compress bound each).
    decompress: ``streams`` = list of (uint8 tensor, size, header bytes)."""

    def __init__(self, ctx: Context, fields=None, streams=None):
        import torch
        self.ctx = ctx
        self.handle = 0
        ctx._children.add(self)
        self._keep = []
        h = ctypes.c_void_p(0)
        if fields is not None:
            n = len(fields)
            descs = (hpez_field_desc * n)()
            self.outs = []
            for i, (x, eb, mode, cfg) in enumerate(fields):
                assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
                cap = hpez_compress_bound(tuple(x.shape))
                out = torch.empty(cap, dtype=torch.uint8, device=x.device)
                self.outs.append(out)
                d = descs[i]
                d.d_in = x.data_ptr()
                d.ndim = x.dim()
                d.eb_mode = mode
                for k in range(3):
                    d.dims[k] = int(x.shape[k]) if k < x.dim() else 1
                d.eb = float(eb)
                if cfg is not None:
                    self._keep.append(cfg)
                    d.cfg = ctypes.pointer(cfg)
                d.d_out = out.data_ptr()
                d.out_cap = cap
            self._keep.append(descs)
            _check(_load().hpez_batch_create_compress(ctx.handle, n, descs, ctypes.byref(h)),
                   "hpez_batch_create_compress")
            self.decomp = False
        else:
            n = len(streams)
            descs = (hpez_stream_desc * n)()
            self.outs = []
            for i, (buf, size, header) in enumerate(streams):
                _, shape, _ = hpez_inspect(header)
                out = torch.empty(shape, dtype=torch.float32, device=buf.device)
                self.outs.append(out)
                hb = np.frombuffer(header[:HPEZ_HEADER_BYTES], dtype=np.uint8).copy()
                self._keep.append(hb)
                d = descs[i]
                d.d_in = buf.data_ptr()
                d.in_size = size
                d.h_header = hb.ctypes.data
                d.d_out = out.data_ptr()
                d.out_cap_elems = out.numel()
            self._keep.append(descs)
            _check(_load().hpez_batch_create_decompress(ctx.handle, n, descs, ctypes.byref(h)),
                   "hpez_batch_create_decompress")
            self.decomp = True
        self.n = n
        self.handle = h.value

    def run(self, stream=None, graph=False):
        s = Context._stream(stream)
        if graph:
            _check(_load().hpez_batch_run_graph(self.handle, s), "hpez_batch_run_graph")
        else:
            _check(_load().hpez_batch_run(self.handle, s), "hpez_batch_run")

    def results(self, stream=None):
        sizes = (ctypes.c_uint64 * self.n)()
        status = (ctypes.c_int32 * self.n)()
        _check(_load().hpez_batch_results(self.handle, Context._stream(stream), sizes, status),
               "hpez_batch_results")
        return list(sizes), list(status)

    def launch_count(self):
        a, b = ctypes.c_uint64(0), ctypes.c_uint64(0)
        _check(_load().hpez_batch_launch_count(self.handle, ctypes.byref(a), ctypes.byref(b)),
               "hpez_batch_launch_count")
        return a.value, b.value

    def close(self):
        if self.handle:
            _load().hpez_batch_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The served form: submit requests with host buffers, step, poll."""

    def __init__(self, ctx: Context, budget_bytes: int, max_slots: int = 64,
                 stream=None):
        import torch
        self.ctx = ctx
        self.handle = 0
        ctx._children.add(self)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = ctypes.c_void_p(0)
        _check(_load().hpez_server_create(ctx.handle, int(budget_bytes), max_slots,
                                          self.stream.cuda_stream, ctypes.byref(h)),
               "hpez_server_create")
        self.handle = h.value
        self._keep = {}

    def submit_compress(self, h_in: np.ndarray, eb: float, eb_mode=HPEZ_EB_REL,
                        cfg=None, h_out=None):
        """h_in: C-contiguous float32 (pinned memory for asynchronous copies).
        Returns (id, output buffer)."""
        assert h_in.dtype == np.float32 and h_in.flags.c_contiguous
        if h_out is None:
            h_out = np.empty(hpez_compress_bound(h_in.shape), dtype=np.uint8)
        r = hpez_request()
        r.op = HPEZ_REQ_COMPRESS
        r.ndim = h_in.ndim
        for k in range(3):
            r.dims[k] = int(h_in.shape[k]) if k < h_in.ndim else 1
        r.eb_mode = eb_mode
        r.eb = float(eb)
        if cfg is not None:
            r.cfg = ctypes.pointer(cfg)
        r.h_in = h_in.ctypes.data
        r.h_out = h_out.ctypes.data
        r.out_cap = h_out.nbytes
        rid = ctypes.c_uint64(0)
        _check(_load().hpez_server_submit(self.handle, ctypes.byref(r), ctypes.byref(rid)),
               "hpez_server_submit")
        self._keep[rid.value] = (h_in, h_out, cfg)
        return rid.value, h_out

    def submit_decompress(self, h_stream: np.ndarray, size: int, h_out=None):
        _, shape, _ = hpez_inspect(h_stream[:HPEZ_HEADER_BYTES].tobytes())
        if h_out is None:
            h_out = np.empty(shape, dtype=np.float32)
        r = hpez_request()
        r.op = HPEZ_REQ_DECOMPRESS
        r.h_in = h_stream.ctypes.data
        r.in_bytes = int(size)
        r.h_out = h_out.ctypes.data
        r.out_cap = h_out.nbytes
        rid = ctypes.c_uint64(0)
        _check(_load().hpez_server_submit(self.handle, ctypes.byref(r), ctypes.byref(rid)),
               "hpez_server_submit")
        self._keep[rid.value] = (h_stream, h_out, None)
        return rid.value, h_out

    def step(self):
        _check(_load().hpez_server_step(self.handle), "hpez_server_step")

    def poll(self, cap: int = 256):
        ids = (ctypes.c_uint64 * cap)()
        st = (ctypes.c_int32 * cap)()
        sz = (ctypes.c_uint64 * cap)()
        lat = (ctypes.c_double * cap)()
        n = ctypes.c_int(0)
        _check(_load().hpez_server_poll(self.handle, cap, ids, st, sz, lat, ctypes.byref(n)),
               "hpez_server_poll")
        out = []
        for i in range(n.value):
            self._keep.pop(ids[i], None)
            out.append((ids[i], st[i], sz[i], lat[i]))
        return out

    def stats(self):
        a, q = ctypes.c_int(0), ctypes.c_int(0)
        u, t, l = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
        _check(_load().hpez_server_stats(self.handle, ctypes.byref(a), ctypes.byref(q),
                                         ctypes.byref(u), ctypes.byref(t), ctypes.byref(l)),
               "hpez_server_stats")
        return dict(active=a.value, queued=q.value, used_bytes=u.value, ticks=t.value,
                    launches=l.value)

    def close(self):
        if self.handle:
            _load().hpez_server_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
