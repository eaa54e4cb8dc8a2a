"""Pins of the oracle's quality-metric target (Sec. 3.1, Eq. 1 with M = PSNR)
and of its integer inputs.

The PSNR is checked against closed forms and a float64 numpy computation;
the bound search against a restatement in Python of its definition (built
on the separately pinned tune / compress / decompress); the integer path
against the error bound it promises, losslessness below 1, the types'
ranges and its refusals.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_12133_gb300 import fields


def test_psnr_closed_forms():
    rng = np.random.default_rng(0)
    unit = 2.0 ** -10
    x = (np.rint(rng.uniform(-3, 5, 4096) / unit) * unit).astype(np.float32)
    k = rng.integers(-200, 201, x.size)
    # errors that are exact multiples of the unit: the MSE is exact
    y = (x.astype(np.float64) - k * unit).astype(np.float32)
    assert np.all((x.astype(np.float64) - y.astype(np.float64)) / unit == k)
    ps, sse = O.psnr(x, y, unit)
    assert sse == int(np.sum(k.astype(np.int64) ** 2))
    rngv = float(x.max()) - float(x.min())
    want = 20 * math.log10(rngv) - 10 * math.log10(sse * unit * unit / x.size)
    assert ps == pytest.approx(want, rel=1e-14)
    assert O.psnr(x, x.copy(), unit)[0] == math.inf


def test_psnr_against_float64():
    """Errors anywhere in [-e, e]: the fixed-point sum is within the
    rounding of 2^-16 e per point of the float64 PSNR."""
    x = fields.grf((40, 50, 60), seed=3).ravel()
    e = 1e-3 * float(x.max() - x.min())
    d = np.random.default_rng(1).uniform(-e, e, x.size)
    y = (x.astype(np.float64) + d).astype(np.float32)
    dd = x.astype(np.float64) - y.astype(np.float64)
    want = 20 * math.log10(float(x.max()) - float(x.min())) - 10 * math.log10(np.mean(dd * dd))
    assert O.psnr(x, y, np.float32(e) / 65536.0)[0] == pytest.approx(want, abs=1e-3)
    # uniform errors on [-e, e] have MSE e^2 / 3
    uni = 20 * math.log10(float(x.max()) - float(x.min())) - 10 * math.log10(e * e / 3)
    assert O.psnr(x, y, e / 65536.0)[0] == pytest.approx(uni, abs=0.05)


def _psnr_fixed(x, y, unit):
    """The metric restated: squared errors in the fixed-point unit."""
    q = np.rint((x.astype(np.float64).ravel() - y.astype(np.float64).ravel()) / unit)
    sse = int(np.sum(q.astype(np.int64) ** 2))
    if sse == 0:
        return math.inf
    r = float(x.max()) - float(x.min())
    return 20.0 * math.log10(r) - 10.0 * math.log10(sse * unit * unit / x.size)


def _search(x, target):
    """The bound search restated from its definition (bracket by doubling or
    halving from the uniform-error bound, 8 geometric bisection steps)."""
    def probe(e):
        cfg, _ = O.tune(x, e, O.EB_ABS)
        s, st, _, _ = O.compress(x, e, O.EB_ABS, cfg)
        y = O.decompress(s)
        return _psnr_fixed(x, y, float(st.e) / 65536.0), s
    rng = float(x.max()) - float(x.min())
    e = rng * math.sqrt(3.0) * 10 ** (-target / 20.0)
    p, _ = probe(e)
    if p >= target:
        lo, hi = e, 2 * e
        for _ in range(6):
            if probe(hi)[0] < target:
                break
            lo, hi = hi, 2 * hi
        else:
            hi = None
    else:
        hi, lo = e, e / 2
        for _ in range(6):
            if probe(lo)[0] >= target:
                break
            hi, lo = lo, lo / 2
        else:
            hi, lo = None, 2 * lo
    if hi is not None:
        for _ in range(8):
            mid = math.sqrt(lo * hi)
            if probe(mid)[0] >= target:
                lo = mid
            else:
                hi = mid
    p, s = probe(lo)
    return s, lo, p, hi


@pytest.mark.parametrize("kind,shape,target", [("grf", (24, 28, 32), 60.0),
                                               ("bumps", (30, 26, 20), 80.0),
                                               ("climate2d", (60, 90), 70.0)])
def test_psnr_target_is_the_search(kind, shape, target):
    x = fields.make(kind, shape, 5)
    s, e, p = O.compress_psnr(x, target)
    ws, we, wp, hi = _search(x, target)
    assert e == we and s == ws and p == wp
    assert p >= target
    # the bound is the largest the search could keep: the failing end of
    # the final bracket lies within a 2^(1/256) factor
    assert hi is not None and hi / e <= 2.0 ** (1 / 256) * 1.0000001
    y = O.decompress(s)
    assert np.all(np.abs(y.astype(np.float64) - x) <= np.float32(e))


def test_psnr_target_refuses_nonfinite():
    x = fields.grf((10, 10, 10), seed=1)
    x[3, 3, 3] = np.nan
    with pytest.raises(O.OracleError):
        O.compress_psnr(x, 60.0)


@pytest.mark.parametrize("dtype,scale,off", [(np.int16, 3000, 0), (np.uint16, 20000, 30000),
                                             (np.int32, 1e6, -5e5)])
@pytest.mark.parametrize("eb", [0.4, 1.0, 7.5])
def test_integer_round_trip_bound(dtype, scale, off, eb):
    x = np.rint(fields.bumps((20, 24, 28), seed=2) * scale + off).astype(dtype)
    s = O.compress_typed(x, eb, O.EB_ABS)
    y = O.decompress_typed(s, dtype)
    err = np.abs(y.astype(np.int64) - x.astype(np.int64))
    assert err.max() <= math.floor(eb)
    if eb < 1:
        assert np.array_equal(y, x)
    # the stream's float bound keeps rounding inside the integer bound
    _, _, abs_eb = O.inspect(s)
    assert np.float32(abs_eb) == np.nextafter(np.float32(math.floor(eb) + 0.5),
                                              np.float32(0))
    assert np.frombuffer(s[O.H_DTYPE:O.H_DTYPE + 4], np.uint32)[0] == \
        {np.int16: O.DTYPE_I16, np.uint16: O.DTYPE_U16, np.int32: O.DTYPE_I32}[dtype]


def test_integer_clamps_and_relative_bound():
    """Values at the ends of the type stay in range; a relative bound is
    taken on the integer value range; auto-tuning keeps the bound."""
    rng = np.random.default_rng(4)
    x = np.zeros((30, 40), np.uint16)
    x[:, :20] = 0
    x[:, 20:] = 65535
    x += rng.integers(0, 3, x.shape).astype(np.uint16) * (x == 0)
    s = O.compress_typed(x, 9.0, O.EB_ABS)
    y = O.decompress_typed(s, np.uint16)
    assert np.abs(y.astype(int) - x.astype(int)).max() <= 9
    z = np.rint(fields.grf((16, 18, 20), seed=6) * 500).astype(np.int16)
    s = O.compress_typed(z, 1e-2, O.EB_REL, tune=True)
    w = O.decompress_typed(s, np.int16)
    assert np.abs(w.astype(int) - z.astype(int)).max() <= math.floor(
        1e-2 * (int(z.max()) - int(z.min())))


def test_integer_refusals():
    x = np.array([[0, 1 << 25]], np.int32)
    with pytest.raises(O.OracleError):
        O.compress_typed(x, 1.0)
    s = O.compress_typed(np.arange(100, dtype=np.int16).reshape(10, 10), 1.0)
    with pytest.raises(O.OracleError):
        O.decompress_typed(s, np.uint16)
