"""ctypes wrapper of the HPEZ CPU oracle (``hpez_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  The product
path (the CUDA library and its binding) never imports, links or executes
anything under ``oracle/``.

The oracle is a plain single-threaded C restatement of the paper's method
(arXiv 2311.12133, Sec. 4-6), compiled as strict IEEE binary32
(``-ffp-contract=off``, no fast-math), and pinned by the ``-m "not gpu"``
tests against closed forms, dense spline solves, brute force and invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hpez_oracle.c")
_HDR = os.path.join(_HERE, "hpez_oracle.h")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD_DIR, "libhpez_oracle.so")
_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fno-unsafe-math-optimizations", "-fPIC", "-shared", "-Wall"]

MAX_LEVELS = 16
RADIUS = 32768
LINEAR, CUBIC_NAK, CUBIC_NAT, SPLINE_GLOBAL = 0, 1, 2, 3
P1D, PMD = 0, 1
EB_ABS, EB_REL = 0, 1

ERRORS = {0: "ok", -1: "invalid argument", -2: "non-finite input",
          -3: "output too small", -4: "corrupt stream", -5: "no memory",
          -6: "self-check failed"}


class OracleError(RuntimeError):
    def __init__(self, rc: int):
        super().__init__(f"oracle error {rc}: {ERRORS.get(rc, '?')}")
        self.rc = rc


class Config(ctypes.Structure):
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
        ("interp", ctypes.c_uint8 * MAX_LEVELS),
        ("paradigm", ctypes.c_uint8 * MAX_LEVELS),
        ("same_level", ctypes.c_uint8 * MAX_LEVELS),
        ("order", (ctypes.c_uint8 * 3) * MAX_LEVELS),
        ("blockmap", ctypes.c_void_p),
    ]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "n_points", "n_anchors", "n_outliers", "n_used", "total_words",
        "n_chunks", "predicted", "bad_reads", "double_visits",
        "sum_len_bits")] + [("e", ctypes.c_float), ("vmin", ctypes.c_float),
                            ("vmax", ctypes.c_float)]


class TuneParams(ctypes.Structure):
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


class TuneReport(ctypes.Structure):
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
        ("level_choice", (ctypes.c_uint8 * MAX_LEVELS) * 2),
        ("level_score", (ctypes.c_uint64 * MAX_LEVELS) * 2),
    ]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, strict IEEE flags)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u64p = ctypes.POINTER(ctypes.c_uint64)
            L.ora_compress.restype = ctypes.c_int
            L.ora_compress.argtypes = [
                ctypes.c_void_p, ctypes.c_int, u64p, ctypes.c_int,
                ctypes.c_double, ctypes.POINTER(Config), ctypes.c_void_p,
                ctypes.c_uint64, u64p, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.POINTER(Stats)]
            L.ora_decompress.restype = ctypes.c_int
            L.ora_decompress.argtypes = [ctypes.c_void_p, ctypes.c_uint64,
                                         ctypes.c_void_p, ctypes.c_uint64]
            L.ora_compress_bound.restype = ctypes.c_uint64
            L.ora_compress_bound.argtypes = [ctypes.c_int, u64p]
            L.ora_default_config.restype = None
            L.ora_default_config.argtypes = [ctypes.c_int,
                                             ctypes.POINTER(Config)]
            L.ora_predict_1d.restype = ctypes.c_float
            L.ora_predict_1d.argtypes = [ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.c_uint64]
            L.ora_quantize.restype = ctypes.c_uint16
            L.ora_quantize.argtypes = [ctypes.c_float] * 5 + [
                ctypes.POINTER(ctypes.c_float)]
            L.ora_level_params.restype = ctypes.c_int
            L.ora_level_params.argtypes = [
                ctypes.c_float, ctypes.c_double, ctypes.c_double,
                ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_void_p]
            L.ora_huffman_lengths.restype = ctypes.c_int
            L.ora_huffman_lengths.argtypes = [ctypes.c_void_p, ctypes.c_int,
                                              ctypes.c_void_p]
            L.ora_canonical_codes.restype = ctypes.c_int
            L.ora_canonical_codes.argtypes = [ctypes.c_void_p, ctypes.c_int,
                                              ctypes.c_void_p]
            L.ora_md_weight.restype = ctypes.c_float
            L.ora_md_weight.argtypes = [ctypes.c_void_p, ctypes.c_uint,
                                        ctypes.c_int]
            L.ora_inspect.restype = ctypes.c_int
            L.ora_inspect.argtypes = [ctypes.c_void_p, ctypes.c_uint64,
                                      ctypes.POINTER(ctypes.c_int), u64p,
                                      ctypes.POINTER(ctypes.c_double)]
            L.ora_default_tune_params.restype = None
            L.ora_default_tune_params.argtypes = [ctypes.POINTER(TuneParams)]
            L.ora_blockmap_size.restype = ctypes.c_uint64
            L.ora_blockmap_size.argtypes = [ctypes.c_int, u64p, ctypes.c_int]
            L.ora_tune.restype = ctypes.c_int
            L.ora_tune.argtypes = [
                ctypes.c_void_p, ctypes.c_int, u64p, ctypes.c_int,
                ctypes.c_double, ctypes.POINTER(TuneParams),
                ctypes.POINTER(Config), ctypes.c_void_p, ctypes.c_uint64,
                ctypes.POINTER(TuneReport)]
            L.ora_tune_candidate.restype = ctypes.c_int
            L.ora_tune_candidate.argtypes = [
                ctypes.POINTER(TuneParams), ctypes.c_int, ctypes.c_int,
                ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                ctypes.POINTER(ctypes.c_int), ctypes.c_void_p,
                ctypes.POINTER(ctypes.c_int)]
            L.ora_subfield_test.restype = ctypes.c_int
            L.ora_subfield_test.argtypes = [
                ctypes.c_void_p, ctypes.c_int, u64p, ctypes.POINTER(Config),
                ctypes.c_float, ctypes.c_int, ctypes.c_void_p,
                ctypes.c_void_p, u64p, u64p]
            L.ora_psnr.restype = ctypes.c_int
            L.ora_psnr.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                   ctypes.c_double, ctypes.POINTER(ctypes.c_double), u64p]
            L.ora_compress_psnr.restype = ctypes.c_int
            L.ora_compress_psnr.argtypes = [
                ctypes.c_void_p, ctypes.c_int, u64p, ctypes.c_double,
                ctypes.POINTER(TuneParams), ctypes.c_void_p, ctypes.c_uint64, u64p,
                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
            L.ora_compress_typed.restype = ctypes.c_int
            L.ora_compress_typed.argtypes = [
                ctypes.c_void_p, ctypes.c_int, ctypes.c_int, u64p, ctypes.c_int,
                ctypes.c_double, ctypes.POINTER(Config), ctypes.c_int,
                ctypes.POINTER(TuneParams), ctypes.c_void_p, ctypes.c_uint64, u64p]
            L.ora_decompress_typed.restype = ctypes.c_int
            L.ora_decompress_typed.argtypes = [ctypes.c_void_p, ctypes.c_uint64,
                                               ctypes.c_void_p, ctypes.c_int,
                                               ctypes.c_uint64]
            for f in (L.ora_lossless_encode, L.ora_lossless_decode):
                f.restype = ctypes.c_int
                f.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                              ctypes.c_uint64, u64p]
            _lib = L
    return _lib


def default_config(ndim: int) -> Config:
    c = Config()
    lib().ora_default_config(ndim, ctypes.byref(c))
    return c


def make_config(ndim: int, *, anchor_stride=None, frozen_dim=-1,
                chunk_syms=16384, alpha=1.0, beta=1.0, md_inv_var=(1, 1, 1),
                interp=CUBIC_NAK, paradigm=P1D, same_level=0, order=None,
                blockmap=None, block_size=32, predictor=0) -> Config:
    """Config with one setting for every level unless per-level lists are
    given (index l-1)."""
    c = default_config(ndim)
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

    for l in range(MAX_LEVELS):
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
    c.blockwise = 0
    c.block_size = block_size
    c.predictor = predictor
    c._blockmap_ref = None
    if blockmap is not None:
        bm = np.ascontiguousarray(blockmap, dtype=np.uint8)
        c._blockmap_ref = bm
        c.blockmap = bm.ctypes.data
        c.blockwise = 1
    return c


def compress(x: np.ndarray, eb: float, eb_mode: int = EB_REL,
             config: Config | None = None, want_codes=False,
             want_recon=False):
    """Returns (stream bytes, stats, codes or None, recon or None)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    ndim = x.ndim
    dims = (ctypes.c_uint64 * 3)(*[int(v) for v in x.shape] + [1] * (3 - ndim))
    L = lib()
    cap = int(L.ora_compress_bound(ndim, dims))
    out = np.zeros(cap, dtype=np.uint8)
    size = ctypes.c_uint64(0)
    st = Stats()
    codes = np.zeros(x.size, dtype=np.uint16) if want_codes else None
    recon = np.zeros(x.size, dtype=np.float32) if want_recon else None
    rc = L.ora_compress(
        x.ctypes.data, ndim, dims, eb_mode, float(eb),
        ctypes.byref(config) if config is not None else None,
        out.ctypes.data, cap, ctypes.byref(size),
        codes.ctypes.data if codes is not None else None,
        recon.ctypes.data if recon is not None else None, ctypes.byref(st))
    if rc != 0:
        raise OracleError(rc)
    return (out[:size.value].tobytes(), st,
            codes.reshape(x.shape) if codes is not None else None,
            recon.reshape(x.shape) if recon is not None else None)


def inspect(stream: bytes):
    buf = np.frombuffer(stream, dtype=np.uint8)
    nd = ctypes.c_int(0)
    dims = (ctypes.c_uint64 * 3)()
    eb = ctypes.c_double(0)
    rc = lib().ora_inspect(buf.ctypes.data, len(stream), ctypes.byref(nd),
                           dims, ctypes.byref(eb))
    if rc != 0:
        raise OracleError(rc)
    return nd.value, tuple(int(dims[i]) for i in range(nd.value)), eb.value


def decompress(stream: bytes) -> np.ndarray:
    nd, shape, _ = inspect(stream)
    buf = np.frombuffer(stream, dtype=np.uint8)
    out = np.zeros(int(np.prod(shape)), dtype=np.float32)
    rc = lib().ora_decompress(buf.ctypes.data, len(stream), out.ctypes.data,
                              out.size)
    if rc != 0:
        raise OracleError(rc)
    return out.reshape(shape)


def predict_1d(kind: int, half_b: int, line: np.ndarray, pos: int,
               s: int) -> np.float32:
    line = np.ascontiguousarray(line, dtype=np.float32)
    return np.float32(lib().ora_predict_1d(kind, half_b, line.ctypes.data,
                                           line.size, pos, s))


def quantize(x, p, el, inv2, twoe):
    r = ctypes.c_float(0)
    code = lib().ora_quantize(float(x), float(p), float(el), float(inv2),
                              float(twoe), ctypes.byref(r))
    return int(code), np.float32(r.value)


def level_params(e: float, alpha: float, beta: float, L: int):
    el = np.zeros(L, np.float32)
    inv2 = np.zeros(L, np.float32)
    twoe = np.zeros(L, np.float32)
    rc = lib().ora_level_params(float(e), float(alpha), float(beta), L,
                                el.ctypes.data, inv2.ctypes.data,
                                twoe.ctypes.data)
    if rc != 0:
        raise OracleError(rc)
    return el, inv2, twoe


def huffman_lengths(freq) -> np.ndarray:
    f = np.ascontiguousarray(freq, dtype=np.uint64)
    lens = np.zeros(f.size, np.uint8)
    rc = lib().ora_huffman_lengths(f.ctypes.data, f.size, lens.ctypes.data)
    if rc != 0:
        raise OracleError(rc)
    return lens


def canonical_codes(lens) -> np.ndarray:
    ln = np.ascontiguousarray(lens, dtype=np.uint8)
    codes = np.zeros(ln.size, np.uint64)
    rc = lib().ora_canonical_codes(ln.ctypes.data, ln.size, codes.ctypes.data)
    if rc != 0:
        raise OracleError(rc)
    return codes


def md_weight(inv_var, mask: int, d: int) -> np.float32:
    iv = np.ascontiguousarray(inv_var, dtype=np.float64)
    return np.float32(lib().ora_md_weight(iv.ctypes.data, mask, d))


# ---------------------------------------------------------------- tuning
def default_tune_params(**kw) -> TuneParams:
    t = TuneParams()
    lib().ora_default_tune_params(ctypes.byref(t))
    for k, v in kw.items():
        setattr(t, k, v)
    return t


def blockmap_size(shape, block_size: int = 32) -> int:
    dims = (ctypes.c_uint64 * 3)(*[int(v) for v in shape] + [1] * (3 - len(shape)))
    return int(lib().ora_blockmap_size(len(shape), dims, block_size))


def tune(x: np.ndarray, eb: float, eb_mode: int = EB_REL,
         params: TuneParams | None = None):
    """Runs the Sec. 6 tuner; returns (config, report).  The config keeps a
    reference to its block map when one was produced."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    ndim = x.ndim
    dims = (ctypes.c_uint64 * 3)(*[int(v) for v in x.shape] + [1] * (3 - ndim))
    tp = params if params is not None else default_tune_params()
    nbm = blockmap_size(x.shape, tp.block_size)
    bm = np.zeros(max(nbm, 1), np.uint8)
    cfg = Config()
    rep = TuneReport()
    rc = lib().ora_tune(x.ctypes.data, ndim, dims, eb_mode, float(eb),
                        ctypes.byref(tp), ctypes.byref(cfg), bm.ctypes.data,
                        bm.size, ctypes.byref(rep))
    if rc != 0:
        raise OracleError(rc)
    cfg._blockmap_ref = bm[:nbm] if cfg.blockwise else None
    if cfg.blockwise:
        cfg.blockmap = cfg._blockmap_ref.ctypes.data
    return cfg, rep


def tune_candidate(ndim: int, frozen: int, j: int,
                   params: TuneParams | None = None):
    """(kind, paradigm, order tuple, same_level) of candidate j, or None."""
    tp = params if params is not None else default_tune_params()
    kind, par, same = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    order = (ctypes.c_uint8 * 3)()
    ok = lib().ora_tune_candidate(ctypes.byref(tp), ndim, frozen, j,
                                  ctypes.byref(kind), ctypes.byref(par),
                                  order, ctypes.byref(same))
    if not ok:
        return None
    return kind.value, par.value, tuple(order), same.value


def subfield_test(xs: np.ndarray, config: Config, e: float, l_stop: int = 1):
    """Compression test on a sub-field: (scores[16], hist, n_out, n_anchors)."""
    xs = np.ascontiguousarray(xs, dtype=np.float32)
    ndim = xs.ndim
    dims = (ctypes.c_uint64 * 3)(*[int(v) for v in xs.shape] + [1] * (3 - ndim))
    score = np.zeros(MAX_LEVELS, np.uint64)
    hist = np.zeros(65536, np.uint64)
    nout = ctypes.c_uint64(0)
    na = ctypes.c_uint64(0)
    rc = lib().ora_subfield_test(xs.ctypes.data, ndim, dims,
                                 ctypes.byref(config), float(e), l_stop,
                                 score.ctypes.data, hist.ctypes.data,
                                 ctypes.byref(nout), ctypes.byref(na))
    if rc != 0:
        raise OracleError(rc)
    return score, hist, nout.value, na.value


# -------------------------------------------- quality target, integer inputs
DTYPE_F32, DTYPE_I16, DTYPE_U16, DTYPE_I32 = 0, 1, 2, 3
H_DTYPE = 320
_DT = {DTYPE_F32: np.float32, DTYPE_I16: np.int16, DTYPE_U16: np.uint16,
       DTYPE_I32: np.int32}


def psnr(x: np.ndarray, y: np.ndarray, unit: float):
    """(PSNR in dB, fixed-point squared-error sum) of y against x."""
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    y = np.ascontiguousarray(y, dtype=np.float32).ravel()
    out = ctypes.c_double(0)
    sse = ctypes.c_uint64(0)
    rc = lib().ora_psnr(x.ctypes.data, y.ctypes.data, x.size, float(unit),
                        ctypes.byref(out), ctypes.byref(sse))
    if rc != 0:
        raise OracleError(rc)
    return out.value, sse.value


def compress_psnr(x: np.ndarray, target_db: float, params: TuneParams | None = None):
    """Eq. 1 with M = PSNR: (stream, absolute bound, PSNR) of the search."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    dims = (ctypes.c_uint64 * 3)(*[int(v) for v in x.shape] + [1] * (3 - x.ndim))
    cap = int(lib().ora_compress_bound(x.ndim, dims))
    out = np.zeros(cap, np.uint8)
    size = ctypes.c_uint64(0)
    eb = ctypes.c_double(0)
    ps = ctypes.c_double(0)
    rc = lib().ora_compress_psnr(x.ctypes.data, x.ndim, dims, float(target_db),
                                 ctypes.byref(params) if params is not None else None,
                                 out.ctypes.data, cap, ctypes.byref(size), ctypes.byref(eb),
                                 ctypes.byref(ps))
    if rc != 0:
        raise OracleError(rc)
    return out[:size.value].tobytes(), eb.value, ps.value


def compress_typed(x: np.ndarray, eb: float, eb_mode: int = EB_ABS,
                   config: Config | None = None, tune: bool = False,
                   params: TuneParams | None = None) -> bytes:
    """Integer (int16, uint16, int32) or float input; the stream."""
    dt = {np.dtype(v): k for k, v in _DT.items()}[np.dtype(x.dtype)]
    x = np.ascontiguousarray(x)
    dims = (ctypes.c_uint64 * 3)(*[int(v) for v in x.shape] + [1] * (3 - x.ndim))
    cap = int(lib().ora_compress_bound(x.ndim, dims))
    out = np.zeros(cap, np.uint8)
    size = ctypes.c_uint64(0)
    rc = lib().ora_compress_typed(x.ctypes.data, dt, x.ndim, dims, eb_mode, float(eb),
                                  ctypes.byref(config) if config is not None else None,
                                  int(tune),
                                  ctypes.byref(params) if params is not None else None,
                                  out.ctypes.data, cap, ctypes.byref(size))
    if rc != 0:
        raise OracleError(rc)
    return out[:size.value].tobytes()


def decompress_typed(stream: bytes, dtype) -> np.ndarray:
    dt = {np.dtype(v): k for k, v in _DT.items()}[np.dtype(dtype)]
    nd, shape, _ = inspect(stream)
    buf = np.frombuffer(stream, dtype=np.uint8)
    out = np.zeros(int(np.prod(shape)), dtype=_DT[dt])
    rc = lib().ora_decompress_typed(buf.ctypes.data, len(stream), out.ctypes.data, dt,
                                    out.size)
    if rc != 0:
        raise OracleError(rc)
    return out.reshape(shape)


# ------------------------------------------------------- the lossless stage
H_RAWSIZE = 328


def lossless_encode(stream: bytes) -> bytes:
    src = np.frombuffer(stream, np.uint8).copy()
    out = np.zeros(len(stream) + 64, np.uint8)
    size = ctypes.c_uint64(0)
    rc = lib().ora_lossless_encode(src.ctypes.data, len(stream), out.ctypes.data, out.size,
                                   ctypes.byref(size))
    if rc != 0:
        raise OracleError(rc)
    return out[:size.value].tobytes()


def lossless_decode(z: bytes) -> bytes:
    src = np.frombuffer(z, np.uint8)
    raw = int.from_bytes(z[H_RAWSIZE:H_RAWSIZE + 8], "little")
    out = np.zeros(max(raw, 1), np.uint8)
    size = ctypes.c_uint64(0)
    rc = lib().ora_lossless_decode(src.ctypes.data, len(z), out.ctypes.data, out.size,
                                   ctypes.byref(size))
    if rc != 0:
        raise OracleError(rc)
    return out[:size.value].tobytes()
