"""Pins of the oracle's global natural-spline interpolator (interp id 3):
along each pass line, the natural cubic spline through every known point of
the line (the knots at multiples of 2s), evaluated halfway between knots.
The paper's Eq. 6 is a local four-knot spline; this is the whole-line form.

Expected values come from outside the oracle: scipy's natural CubicSpline
in double precision, run level by level on the reconstruction it implies,
and the exactness of a spline on linear data.  With an error bound far
above the data's spread every code is the zero quantum, so the
reconstruction is the prediction itself and can be compared point by point.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_12133_gb300 import fields

scipy_interp = pytest.importorskip("scipy.interpolate")
R = 32768


def _line_levels(line, A):
    """Double-precision reference of the sweep along one line (1D field):
    anchors at multiples of A, then per level the natural spline through
    the known points at the midpoints; no right knot: (3 y_K - y_{K-1}) / 2,
    or y_K with a single knot."""
    n = len(line)
    rec = np.full(n, np.nan)
    rec[::A] = line[::A]
    s = A // 2
    while s >= 1:
        kpos = np.arange(0, n, 2 * s)
        kval = rec[kpos]
        mids = np.arange(s, n, 2 * s)
        if len(kpos) >= 2:
            cs = scipy_interp.CubicSpline(kpos, kval, bc_type="natural")
        for m in mids:
            if m + s <= n - 1:
                rec[m] = cs(m)
            elif len(kpos) >= 2:
                rec[m] = (3 * kval[-1] - kval[-2]) / 2
            else:
                rec[m] = kval[-1]
        s //= 2
    return rec


@pytest.mark.parametrize("n,A", [(129, 32), (200, 64), (37, 8), (5, 4), (2, 2), (1000, 128)])
def test_1d_matches_natural_spline(n, A):
    rng = np.random.default_rng(n)
    x = np.cumsum(rng.normal(0, 1, n)).astype(np.float32)
    c = O.make_config(1, anchor_stride=A, interp=O.SPLINE_GLOBAL)
    s, st, codes, rec = O.compress(x, 1e6, O.EB_ABS, c, want_codes=True, want_recon=True)
    assert np.all(codes == R)
    want = _line_levels(x.astype(np.float64), A)
    scale = np.abs(x).max() + 1.0
    assert np.max(np.abs(rec.astype(np.float64) - want)) <= 2e-5 * scale
    assert O.decompress(s).tobytes() == rec.tobytes()


def test_2d_lines_follow_the_pass_order():
    """2D, both 1D-style orders: at each level the first pass splines along
    its dimension on the even rows, the second along the other on every
    row; checked against the double-precision reference pass by pass."""
    rng = np.random.default_rng(3)
    x = rng.normal(0, 1, (33, 47)).astype(np.float32)
    A = 16
    for order in ((0, 1), (1, 0)):
        c = O.make_config(2, anchor_stride=A, interp=O.SPLINE_GLOBAL, order=order)
        _, _, codes, rec = O.compress(x, 1e6, O.EB_ABS, c, want_codes=True, want_recon=True)
        assert np.all(codes == R)
        ref = np.full(x.shape, np.nan)
        ref[::A, ::A] = x[::A, ::A]
        s = A // 2
        while s >= 1:
            known = np.zeros(x.shape, bool)
            known[::2 * s, ::2 * s] = True
            for d in order:
                # lines along d through the points on the stride-s grid whose
                # other coordinate is already known at this level
                other = 1 - d
                for o in range(0, x.shape[other], s):
                    idx = [slice(None), slice(None)]
                    idx[other] = o
                    lk = known[tuple(idx)]
                    if not lk[::2 * s].all():
                        continue
                    line = ref[tuple(idx)]
                    kpos = np.arange(0, x.shape[d], 2 * s)
                    kval = line[kpos]
                    mids = np.arange(s, x.shape[d], 2 * s)
                    cs = (scipy_interp.CubicSpline(kpos, kval, bc_type="natural")
                          if len(kpos) >= 2 else None)
                    for m in mids:
                        if m + s <= x.shape[d] - 1:
                            v = cs(m)
                        elif len(kpos) >= 2:
                            v = (3 * kval[-1] - kval[-2]) / 2
                        else:
                            v = kval[-1]
                        line[m] = v
                        lk[m] = True
                    ref[tuple(idx)] = line
                    known[tuple(idx)] = lk
            s //= 2
        assert not np.isnan(ref).any()
        assert np.max(np.abs(rec.astype(np.float64) - ref)) <= 1e-4


def test_linear_fields_are_exact():
    """A natural spline through points of a linear function is that
    function: every code of an integer-valued linear field is the zero
    quantum, at any bound."""
    i, j, k = np.indices((29, 34, 40))
    x = (3 * i - 2 * j + 5 * k + 7).astype(np.float32)
    for A in (8, 16):
        c = O.make_config(3, anchor_stride=A, interp=O.SPLINE_GLOBAL, order=(2, 0, 1))
        s, st, codes, rec = O.compress(x, 0.01, O.EB_ABS, c, want_codes=True, want_recon=True)
        assert np.all(codes == R)
        assert rec.tobytes() == x.tobytes()


def test_roundtrip_and_level_mix():
    """Global spline on some levels, the local interpolators on others;
    frozen dimension; the error bound holds and the stream round-trips."""
    x = fields.grf((40, 36, 50), seed=2)
    c = O.make_config(3, interp=[O.SPLINE_GLOBAL, O.CUBIC_NAK, O.SPLINE_GLOBAL, O.LINEAR,
                                 O.SPLINE_GLOBAL], frozen_dim=1)
    s, st, _, rec = O.compress(x, 1e-3, O.EB_REL, c, want_recon=True)
    y = O.decompress(s)
    assert y.tobytes() == rec.tobytes()
    assert np.all(np.abs(y.astype(np.float64) - x) <= st.e)
    assert st.bad_reads == 0 and st.double_visits == 0


@pytest.mark.parametrize("kw", [dict(paradigm=1), dict(same_level=1)])
def test_refused_forms(kw):
    x = fields.grf((20, 20), seed=1)
    c = O.make_config(2, interp=O.SPLINE_GLOBAL, **kw)
    with pytest.raises(Exception):
        O.compress(x, 1e-3, O.EB_REL, c)


def test_thomas_coefficients_reach_their_fixed_point():
    """c'_1 = 1/4, c'_k = 1/(4 - c'_{k-1}) in binary32 (IEEE division) is
    stationary from k = 7 on: a table of the first 16 coefficients, reused
    for every larger k, gives each c'_k exactly (the kernel relies on it)."""
    c = [np.float32(0.25)]
    for _ in range(2, 64):
        c.append(np.float32(1.0) / (np.float32(4.0) - c[-1]))
    assert all(v == c[14] for v in c[14:])
    assert c[6] == c[7] and c[5] != c[6]
