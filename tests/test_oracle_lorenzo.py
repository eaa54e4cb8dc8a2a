"""Pins of the oracle's full-field Lorenzo predictor (Sec. 6.5; block-local
reading: blocks of side A, neighbours outside the block read 0) and of the
tuner's choice between it and interpolation.

The expected values come from what the stencils must do, not from the
oracle's code: the order-1 stencil's residual is the mixed difference
D0 D1 D2 x (D the backward difference), so it vanishes inside a block for
any field without a term coupling all three coordinates; the order-2
residual is D0^2 D1^2 D2^2 x, which vanishes for fields linear along one
coordinate in every term; blocks are independent of one another.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_12133_gb300 import fields

R = 32768


def _codes(x, eb, order, A=None):
    kw = dict(predictor=order)
    if A is not None:
        kw["anchor_stride"] = A
    c = O.make_config(x.ndim, **kw)
    s, st, codes, rec = O.compress(x, eb, O.EB_ABS, c, want_codes=True, want_recon=True)
    return s, st, codes, rec


def _interior(shape, A, k):
    """Mask of the points whose block-local coordinates are all >= k."""
    idx = np.indices(shape)
    m = np.ones(shape, bool)
    for d in range(len(shape)):
        m &= (idx[d] % A) >= k
    return m


def test_order1_exact_without_triple_coupling():
    """Integer values with e = 0.5 make every reconstruction exact (a
    residual is an integer, q = the residual, recon = x), so a point's code
    is the zero-error code exactly when the stencil reproduces x."""
    rng = np.random.default_rng(0)
    n = (20, 23, 37)
    # arbitrary (rough) integer functions of two coordinates each
    g = rng.integers(-9, 10, (n[0], n[1]))
    h = rng.integers(-9, 10, (n[1], n[2]))
    u = rng.integers(-9, 10, (n[0], n[2]))
    x = (g[:, :, None] + h[None, :, :] + u[:, None, :]).astype(np.float32)
    _, st, codes, rec = _codes(x, 0.5, 1, A=8)
    assert rec.tobytes() == x.tobytes()
    inner = _interior(n, 8, 1)
    assert np.all(codes[inner] == R)
    # block-border points (the padding reads 0) are not predicted exactly
    assert np.any(codes[~inner] != R)
    # a term coupling all three coordinates breaks it
    i, j, k = np.indices(n)
    y = x + ((i * j * k) % 3 == 0).astype(np.float32)
    _, _, cy, _ = _codes(y, 0.5, 1, A=8)
    assert np.any(cy[inner] != R)


def test_order2_exact_for_linear_terms():
    rng = np.random.default_rng(2)
    n = (18, 19, 40)
    i, j, k = np.indices(n)
    # every term is linear along at least one coordinate
    g = rng.integers(-4, 5, (n[0], n[1]))
    h = rng.integers(-4, 5, (n[1], n[2]))
    u = rng.integers(-4, 5, (n[0], n[2]))
    x = (g[:, :, None] * k + h[None, :, :] * i + u[:, None, :] * j).astype(np.float32)
    _, _, codes, rec = _codes(x, 0.5, 2, A=16)
    assert rec.tobytes() == x.tobytes()
    assert np.all(codes[_interior(n, 16, 2)] == R)
    # order 1 does not predict these exactly
    _, _, c1, _ = _codes(x, 0.5, 1, A=16)
    assert np.any(c1[_interior(n, 16, 2)] != R)


def test_1d_zero_padding_at_block_starts():
    """A constant 1D field: order 1 predicts the constant everywhere but at
    the first point of each block, which reads 0."""
    x = np.full(300, 7.25, np.float32)
    x[0] = 1.0  # not a constant field (REL mode would short-cut; ABS here)
    _, _, codes, rec = _codes(x, 1e-3, 1, A=128)
    starts = np.arange(0, 300, 128)
    mask = np.zeros(300, bool)
    mask[starts] = True
    mask[1] = True  # reads x[0] = 1.0
    assert np.all(codes[~mask] == R)
    assert np.all(codes[starts] != R)
    assert np.all(np.abs(rec.astype(np.float64) - x) <= 1e-3)


@pytest.mark.parametrize("order", [1, 2])
def test_blocks_independent(order):
    x = fields.grf((24, 30, 34), seed=5)
    _, _, c0, _ = _codes(x, 1e-3, order, A=8)
    y = x.copy()
    y[8:16, 8:16, 16:24] += np.float32(0.37)  # one block changed
    _, _, c1, _ = _codes(y, 1e-3, order, A=8)
    diff = c0 != c1
    blk = np.zeros(x.shape, bool)
    blk[8:16, 8:16, 16:24] = True
    assert not np.any(diff & ~blk)
    assert np.any(diff & blk)


@pytest.mark.parametrize("shape,order", [((1000,), 1), ((1000,), 2), ((45, 70), 1),
                                         ((45, 70), 2), ((17, 33, 40), 2)])
def test_roundtrip_bound(shape, order):
    x = fields.grf(shape, seed=len(shape) + order)
    s, st, _, rec = _codes(x, 1e-4, order)
    y = O.decompress(s)
    assert y.tobytes() == rec.tobytes()
    assert np.all(np.abs(y.astype(np.float64) - x) <= st.e)


def test_tuner_selects_lorenzo_when_better():
    """A field Lorenzo predicts exactly inside blocks (no triple coupling)
    and interpolation cannot: the tuner selects Lorenzo, of the order with
    the smaller estimate, and leaves out the block-wise map; with the
    estimate scaled up by a large coefficient it keeps interpolation."""
    rng = np.random.default_rng(1)
    n = (64, 64, 64)
    g = rng.normal(0, 1, (n[0], n[1]))
    h = rng.normal(0, 1, (n[1], n[2]))
    x = (g[:, :, None] + h[None, :, :]).astype(np.float32)
    cfg, rep = O.tune(x, 1e-3, O.EB_REL)
    assert rep.lorenzo_better == 1
    b1, b2 = rep.lorenzo_bits[0], rep.lorenzo_bits[1]
    assert cfg.predictor == (1 if b1 <= b2 else 2)
    assert cfg.blockwise == 0
    s, st, _, _ = O.compress(x, 1e-3, O.EB_REL, cfg)
    y = O.decompress(s)
    assert np.all(np.abs(y.astype(np.float64) - x) <= st.e)
    tp = O.default_tune_params(lorenzo_coef=1e6)
    cfg2, rep2 = O.tune(x, 1e-3, O.EB_REL, tp)
    assert rep2.lorenzo_better == 0 and cfg2.predictor == 0


def test_smooth_field_keeps_interpolation():
    x = fields.grf((64, 64, 64), seed=3)
    cfg, rep = O.tune(x, 1e-3, O.EB_REL)
    assert rep.lorenzo_better == 0 and cfg.predictor == 0
