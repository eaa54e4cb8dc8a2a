"""Seeded synthetic float32 fields shaped like the paper's workloads.

This module holds no compressor arithmetic: it only draws inputs, and both
the CUDA path and the oracle consume the same arrays.  The paper evaluates
on real datasets (Table 1: RTM, SEGSalt, Miranda, SCALE-LetKF, CESM-ATM,
JHTDB); none are available here, so these stand-ins reproduce their shapes
and broad statistics:

* ``bumps``      sum of Gaussian bumps + low-frequency sinusoids + white noise
* ``grf``        Gaussian random field with power spectrum ~ k^slope
                 (slope -5/3: turbulence-like, JHTDB/Miranda stand-in)
* ``lognormal``  exp of a GRF with variance 2 (density-like variant)
* ``aniso``      k^-3 spectrum in the two long dims, white along the short
                 one (SCALE-LetKF stand-in, 98x1200x1200)
* ``climate2d``  latitude-banded mean + k^-3 noise + 5 % constant-fill
                 masked rectangles (CESM-ATM 2D slice stand-in, 1800x3600)

Every generator takes an integer seed and is deterministic (numpy PCG64).
"""
from __future__ import annotations

import hashlib

import numpy as np

try:  # multi-threaded FFT when scipy is present
    import scipy.fft as _fft

    def _rfftn(a, axes=None):
        return _fft.rfftn(a, axes=axes, workers=-1)

    def _irfftn(a, s, axes=None):
        return _fft.irfftn(a, s=s, axes=axes, workers=-1)
except Exception:  # pragma: no cover - numpy fallback
    def _rfftn(a, axes=None):
        return np.fft.rfftn(a, axes=axes)

    def _irfftn(a, s, axes=None):
        return np.fft.irfftn(a, s=s, axes=axes)


def seed_of(*parts) -> int:
    """Stable 63-bit seed from arbitrary printable parts."""
    h = hashlib.sha256("/".join(str(p) for p in parts).encode()).digest()
    return int.from_bytes(h[:8], "little") >> 1


def bumps(shape=(128, 128, 128), seed=0, n_bumps=32, noise=1e-4):
    """Sum of ``n_bumps`` Gaussian bumps (amplitude U(-1,1), width U(4,24)
    cells, centre uniform in the box) + 3 sinusoids (integer wave numbers
    1..3 per axis, random phase, amplitude 0.1) + N(0, noise^2) noise."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    axes = [np.arange(s, dtype=np.float64) for s in shape]
    out = np.zeros(shape, dtype=np.float64)
    for _ in range(n_bumps):
        amp = rng.uniform(-1, 1)
        width = rng.uniform(4, 24)
        ctr = [rng.uniform(0, s) for s in shape]
        g = None
        for d in range(nd):
            gd = np.exp(-0.5 * ((axes[d] - ctr[d]) / width) ** 2)
            sh = [1] * nd
            sh[d] = shape[d]
            gd = gd.reshape(sh)
            g = gd if g is None else g * gd
        out += amp * g
    for _ in range(3):
        k = rng.integers(1, 4, size=nd)
        ph = rng.uniform(0, 2 * np.pi)
        arg = None
        for d in range(nd):
            sh = [1] * nd
            sh[d] = shape[d]
            a = (2 * np.pi * k[d] * axes[d] / shape[d]).reshape(sh)
            arg = a if arg is None else arg + a
        out += 0.1 * np.sin(arg + ph)
    out += rng.normal(0.0, noise, size=shape)
    return out.astype(np.float32)


def _spectral_filter(shape, slope, axes):
    """|k|^(slope/2) amplitude filter over the given axes (rfft layout on
    the last of them); the k=0 mode is removed."""
    ks = []
    for j, ax in enumerate(axes):
        n = shape[ax]
        if j == len(axes) - 1:
            k = np.fft.rfftfreq(n) * n
        else:
            k = np.fft.fftfreq(n) * n
        sh = [1] * len(axes)
        sh[j] = k.size
        ks.append((k.reshape(sh)) ** 2)
    k2 = ks[0]
    for t in ks[1:]:
        k2 = k2 + t
    with np.errstate(divide="ignore"):
        filt = np.where(k2 > 0, k2 ** (slope / 4.0), 0.0)
    return filt


def grf(shape=(128, 128, 128), seed=0, slope=-5.0 / 3.0):
    """Gaussian random field, power spectrum ~ |k|^slope, unit variance."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    w = rng.standard_normal(shape, dtype=np.float32)
    axes = tuple(range(len(shape)))
    W = _rfftn(w, axes=axes)
    del w
    filt = _spectral_filter(shape, slope, axes).astype(np.float32)
    W *= filt
    g = _irfftn(W, s=shape, axes=axes).astype(np.float32, copy=False)
    del W
    g -= g.mean(dtype=np.float64)
    g /= np.float32(g.std(dtype=np.float64))
    return np.ascontiguousarray(g, dtype=np.float32)


def lognormal(shape=(128, 128, 128), seed=0, slope=-5.0 / 3.0, var=2.0):
    """exp(g), g the GRF above scaled to variance ``var``."""
    g = grf(shape, seed, slope)
    g *= np.float32(np.sqrt(var))
    np.exp(g, out=g)
    return g


def aniso(shape=(98, 1200, 1200), seed=0, slope=-3.0):
    """Planes along dim 0 are independent 2D fields with spectrum
    ~ |k|^slope over dims (1, 2): smooth in the long dims, white along the
    short one."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    w = rng.standard_normal(shape, dtype=np.float32)
    W = _rfftn(w, axes=(1, 2))
    del w
    filt = _spectral_filter(shape, slope, (1, 2)).astype(np.float32)
    W *= filt[None]
    g = _irfftn(W, s=shape[1:], axes=(1, 2)).astype(np.float32, copy=False)
    g -= g.mean(dtype=np.float64)
    g /= np.float32(g.std(dtype=np.float64))
    return np.ascontiguousarray(g, dtype=np.float32)


def climate2d(shape=(1800, 3600), seed=0, mask_frac=0.05):
    """Latitude-banded mean (cos of latitude plus bands) + k^-3 noise, with
    rectangular regions covering ~``mask_frac`` of the area set to a constant
    fill (the field minimum), like land masks in ocean fields."""
    rng = np.random.default_rng(seed)
    ny, nx = int(shape[0]), int(shape[1])
    lat = np.linspace(-np.pi / 2, np.pi / 2, ny)
    mean = (30.0 * np.cos(lat) + 3.0 * np.cos(6 * lat)).astype(np.float32)
    noise = grf((ny, nx), seed=seed + 1, slope=-3.0)
    f = mean[:, None] + 2.0 * noise
    fill = np.float32(f.min())
    area = 0
    target = mask_frac * ny * nx
    while area < target:
        h = int(rng.integers(ny // 40, ny // 8))
        w = int(rng.integers(nx // 40, nx // 8))
        y0 = int(rng.integers(0, ny - h))
        x0 = int(rng.integers(0, nx - w))
        f[y0:y0 + h, x0:x0 + w] = fill
        area += h * w
    return np.ascontiguousarray(f, dtype=np.float32)


def grf_torch(shape=(512, 512, 512), seed=0, slope=-5.0 / 3.0, device="cuda"):
    """The ``grf`` recipe drawn on the GPU with torch (same spectrum and
    normalization, different random stream): for large benchmark inputs
    whose host generation would take minutes.  Returns a float32 tensor."""
    import torch
    shape = tuple(int(s) for s in shape)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    w = torch.randn(shape, generator=g, device=device, dtype=torch.float32)
    W = torch.fft.rfftn(w)
    del w
    filt = torch.from_numpy(_spectral_filter(shape, slope,
                                             tuple(range(len(shape))))
                            .astype(np.float32)).to(device)
    W *= filt
    del filt
    f = torch.fft.irfftn(W, s=shape)
    del W
    f -= f.mean(dtype=torch.float64).float()
    f /= f.std().float()
    return f.contiguous()


def _grf_axes_torch(shape, seed, slope, axes, device):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    w = torch.randn(shape, generator=g, device=device, dtype=torch.float32)
    W = torch.fft.rfftn(w, dim=axes)
    del w
    filt = torch.from_numpy(_spectral_filter(shape, slope, axes)
                            .astype(np.float32)).to(device)
    W *= filt
    del filt
    f = torch.fft.irfftn(W, s=[shape[a] for a in axes], dim=axes)
    del W
    f -= f.mean(dtype=torch.float64).float()
    f /= f.std().float()
    return f.contiguous()


def make_torch(kind: str, shape, seed: int, device="cuda"):
    """The recipes above drawn on the GPU with torch (same parameters and
    spectra, a different random stream for the white-noise parts), for
    large or many benchmark inputs.  Returns a float32 CUDA tensor."""
    import torch
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    if kind == "grf":
        return grf_torch(shape, seed, device=device)
    if kind == "lognormal":
        f = grf_torch(shape, seed, device=device)
        f *= float(np.sqrt(2.0))
        return torch.exp_(f)
    if kind == "aniso":
        if nd != 3:
            return grf_torch(shape, seed, slope=-3.0, device=device)
        return _grf_axes_torch(shape, seed, -3.0, (1, 2), device)
    if kind == "bumps":
        rng = np.random.default_rng(seed)
        axes = [torch.arange(n, device=device, dtype=torch.float32) for n in shape]
        out = torch.zeros(shape, device=device, dtype=torch.float32)
        for _ in range(32):
            amp = rng.uniform(-1, 1)
            width = rng.uniform(4, 24)
            ctr = [rng.uniform(0, n) for n in shape]
            g = None
            for d in range(nd):
                gd = torch.exp(-0.5 * ((axes[d] - ctr[d]) / width) ** 2)
                sh = [1] * nd
                sh[d] = shape[d]
                gd = gd.reshape(sh)
                g = gd if g is None else g * gd
            out += amp * g
        for _ in range(3):
            k = rng.integers(1, 4, size=nd)
            ph = rng.uniform(0, 2 * np.pi)
            arg = None
            for d in range(nd):
                sh = [1] * nd
                sh[d] = shape[d]
                a_ = (2 * np.pi * float(k[d]) * axes[d] / shape[d]).reshape(sh)
                arg = a_ if arg is None else arg + a_
            out += 0.1 * torch.sin(arg + ph)
        gen = torch.Generator(device=device)
        gen.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
        out += 1e-4 * torch.randn(shape, generator=gen, device=device)
        return out.contiguous()
    if kind == "climate2d":
        rng = np.random.default_rng(seed)
        ny, nx = shape[-2], shape[-1]
        lat = torch.linspace(-np.pi / 2, np.pi / 2, ny, device=device)
        mean = 30.0 * torch.cos(lat) + 3.0 * torch.cos(6 * lat)
        f = mean[:, None] + 2.0 * grf_torch((ny, nx), seed + 1, slope=-3.0,
                                            device=device)
        fill = float(f.min())
        area, target = 0, 0.05 * ny * nx
        while area < target:
            h = int(rng.integers(max(ny // 40, 1), max(ny // 8, 2)))
            w = int(rng.integers(max(nx // 40, 1), max(nx // 8, 2)))
            y0 = int(rng.integers(0, max(ny - h, 1)))
            x0 = int(rng.integers(0, max(nx - w, 1)))
            f[y0:y0 + h, x0:x0 + w] = fill
            area += h * w
        return f.contiguous()
    raise ValueError(kind)


GENERATORS = {
    "bumps": bumps,
    "grf": grf,
    "lognormal": lognormal,
    "aniso": aniso,
    "climate2d": climate2d,
}


def make(kind: str, shape, seed: int) -> np.ndarray:
    return GENERATORS[kind](tuple(shape), seed)


def batch_mix(n_fields=64, seed=0, lo=32 ** 3, hi=256 * 384 * 384):
    """Per-field (kind, shape, seed, rel eb) for the batched workload: sizes
    log-uniform in [lo, hi] points, about 1/3 2D; generators from the plain
    workloads; relative eb per field from {1e-2, 1e-3, 1e-4}."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_fields):
        npts = float(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        if rng.uniform() < 1.0 / 3.0:
            a = rng.uniform(0.5, 2.0)
            ny = max(8, int(round(np.sqrt(npts / a))))
            nx = max(8, int(round(npts / ny)))
            shape = (ny, nx)
            kind = ["climate2d", "grf"][int(rng.integers(0, 2))]
        else:
            r = rng.uniform(0.5, 2.0, size=3)
            r = r / np.prod(r) ** (1 / 3)
            side = npts ** (1 / 3)
            shape = tuple(max(8, int(round(side * v))) for v in r)
            kind = ["bumps", "grf", "lognormal", "aniso"][int(rng.integers(0, 4))]
        eb = [1e-2, 1e-3, 1e-4][int(rng.integers(0, 3))]
        out.append((kind, shape, seed_of("batch", seed, i), eb))
    return out
