"""Pins of the CPU oracle against what the paper and mathematics fix.

None of these retype the oracle's formulas: stencils are checked against
spline solves (scipy CubicSpline and a dense solve of the Eq. 3 system) and
the printed equations; the quantizer against exact rational arithmetic;
Huffman against a textbook heap construction, the Kraft equality and the
RFC 1951 worked example; the sweep against polynomial reproduction,
coverage/known-before-read self-checks and brute-force round trips.
"""
import heapq
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _weights(oracle, kind, half_b, n, pos, s, offsets, denom):
    """Extract the stencil the oracle applies at `pos` by impulse probing:
    an impulse of height `denom` at each offset (all arithmetic exact)."""
    w = {}
    for off in offsets:
        line = np.zeros(n, np.float32)
        line[pos + off * s] = denom
        w[off] = float(oracle.predict_1d(kind, half_b, line, pos, s)) / denom
    return w


def _spline_weight(knots, bc, at=0.0):
    from scipy.interpolate import CubicSpline
    out = []
    for j in range(len(knots)):
        y = np.zeros(len(knots))
        y[j] = 1.0
        out.append(float(CubicSpline(knots, y, bc_type=bc)(at)))
    return out


def _dense_eq3(bc):
    """Dense solve of the Eq. 3 spline system (3 cubic pieces on knots
    -3,-1,1,3) with either the Eq. 5 not-a-knot or the natural conditions;
    returns the weights of p = f2(0)."""
    knots = [-3.0, -1.0, 1.0, 3.0]
    W = []
    for j in range(4):
        d = np.zeros(4)
        d[j] = 1.0
        A = np.zeros((12, 12))
        b = np.zeros(12)
        r = 0
        # piece k on [knots[k], knots[k+1]]: a(x-x_k)^3 + b(x-x_k)^2 + c(x-x_k) + delta
        def row(k, x, deriv):
            t = x - knots[k]
            v = np.zeros(12)
            if deriv == 0:
                v[4 * k:4 * k + 4] = [t ** 3, t ** 2, t, 1]
            elif deriv == 1:
                v[4 * k:4 * k + 4] = [3 * t ** 2, 2 * t, 1, 0]
            elif deriv == 2:
                v[4 * k:4 * k + 4] = [6 * t, 2, 0, 0]
            else:
                v[4 * k:4 * k + 4] = [6, 0, 0, 0]
            return v
        for k in range(3):
            A[r] = row(k, knots[k], 0); b[r] = d[k]; r += 1
            A[r] = row(k, knots[k + 1], 0); b[r] = d[k + 1]; r += 1
        for k in range(2):
            for der in (1, 2):
                A[r] = row(k, knots[k + 1], der) - row(k + 1, knots[k + 1], der)
                r += 1
        if bc == "not-a-knot":
            for k in range(2):
                A[r] = row(k, knots[k + 1], 3) - row(k + 1, knots[k + 1], 3)
                r += 1
        else:
            A[r] = row(0, knots[0], 2); r += 1
            A[r] = row(2, knots[3], 2); r += 1
        coef = np.linalg.solve(A, b)
        W.append(coef[4 + 3])  # f2(0): piece 1 at t = 0 - (-1) = 1
        t = 1.0
        W[-1] = coef[4] * t ** 3 + coef[5] * t ** 2 + coef[6] * t + coef[7]
    return W


def test_printed_stencils_match_oracle(oracle):
    """Interior stencils equal the equations as printed (golden file)."""
    kinds = {"eq2_linear": (oracle.LINEAR, 0), "eq4_notaknot": (oracle.CUBIC_NAK, 0),
             "eq6_natural": (oracle.CUBIC_NAT, 0),
             "eq10_samelevel": (oracle.CUBIC_NAK, 1),
             "eq11_samelevel": (oracle.CUBIC_NAT, 1)}
    rows = [l for l in open(os.path.join(GOLDEN, "stencils_printed.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 5
    for r in rows:
        name, _, offs, nums, den = [c.strip() for c in r.split("|")]
        offs = [int(v) for v in offs.split()]
        nums = [int(v) for v in nums.split()]
        den = int(den)
        kind, hb = kinds[name]
        for s in (1, 2, 4):
            n, pos = 8 * s + 1, 4 * s  # every neighbour exists
            w = _weights(oracle, kind, hb, n, pos, s, offs, den)
            for o, num in zip(offs, nums):
                assert w[o] == pytest.approx(num / den, abs=0), (name, o)


def test_cubic_stencils_are_spline_solves(oracle):
    """Eq. 4 / Eq. 6 / Eq. 11 are the not-a-knot / natural splines through
    the knots (scipy CubicSpline and a dense solve of Eq. 3)."""
    for kind, bc in ((oracle.CUBIC_NAK, "not-a-knot"), (oracle.CUBIC_NAT, "natural")):
        ref = _spline_weight([-3, -1, 1, 3], bc)
        dense = _dense_eq3(bc)
        w = _weights(oracle, kind, 0, 9, 4, 1, [-3, -1, 1, 3], 80.0)
        got = [w[o] for o in (-3, -1, 1, 3)]
        np.testing.assert_allclose(got, ref, atol=1e-12)
        np.testing.assert_allclose(got, dense, atol=1e-12)
    # Eq. 11: natural spline through the 6 same-level knots
    ref = _spline_weight([-3, -2, -1, 1, 2, 3], "natural")
    w = _weights(oracle, oracle.CUBIC_NAT, 1, 9, 4, 1, [-3, -2, -1, 1, 2, 3], 62.0)
    np.testing.assert_allclose([w[o] for o in (-3, -2, -1, 1, 2, 3)], ref, atol=1e-12)


def test_boundary_fallbacks_are_spline_solves(oracle):
    """With a missing outer knot the stencil is the spline through the
    three available knots (scipy: not-a-knot on 3 knots is the parabola),
    with no right neighbour it is linear extrapolation, else a copy."""
    for kind, bc in ((oracle.CUBIC_NAK, "not-a-knot"), (oracle.CUBIC_NAT, "natural")):
        # d+3 missing: line of length 6 (pos 3, s 1) -> knots -3, -1, 1
        ref = _spline_weight([-3, -1, 1], bc)
        w = _weights(oracle, kind, 0, 5, 3, 1, [-3, -1, 1], 32.0)
        np.testing.assert_allclose([w[-3], w[-1], w[1]], ref, atol=1e-12)
        # d-3 missing: pos 1 -> knots -1, 1, 3
        ref = _spline_weight([-1, 1, 3], bc)
        w = _weights(oracle, kind, 0, 5, 1, 1, [-1, 1, 3], 32.0)
        np.testing.assert_allclose([w[-1], w[1], w[3]], ref, atol=1e-12)
        # both outer knots missing: linear (Eq. 2)
        w = _weights(oracle, kind, 0, 3, 1, 1, [-1, 1], 2.0)
        assert (w[-1], w[1]) == (0.5, 0.5)
        # no right neighbour, d-3 present: line through (-3, d-3), (-1, d-1)
        w = _weights(oracle, kind, 0, 4, 3, 1, [-3, -1], 2.0)
        assert (w[-3], w[-1]) == (-0.5, 1.5)
        # no right neighbour and no d-3: copy d-1
        w = _weights(oracle, kind, 0, 2, 1, 1, [-1], 2.0)
        assert w[-1] == 1.0
    # same-level half with a missing +-2 neighbour falls back to the
    # inter-level stencil of the point
    w = _weights(oracle, oracle.CUBIC_NAK, 1, 5, 3, 1, [-3, -1, 1], 32.0)
    np.testing.assert_allclose([w[-3], w[-1], w[1]],
                               _spline_weight([-3, -1, 1], "not-a-knot"), atol=1e-12)


def _exact_ok(x, r, e):
    return abs(Fraction(float(x)) - Fraction(float(r))) <= Fraction(float(e))


def test_quantizer_bound_and_nearest_code(oracle):
    """Brute force over a small float set: an accepted code always meets
    |x - x'| <= e exactly and is the nearest integer to (x - p)/(2e) (up to
    the rounding of the scaled error); an escape returns x verbatim."""
    vals = np.array([0.0, 1e-7, -1e-7, 0.3, -0.3, 0.5, 0.75, 1.0, -1.0, 1.5,
                     2.0, 3.1, -7.25, 100.0, 1e6, -1e6, 3e38, 1e-38],
                    dtype=np.float32)
    for eb in (np.float32(0.1), np.float32(0.25), np.float32(1e-3), np.float32(3.0)):
        el, inv2, twoe = oracle.level_params(float(eb), 1.0, 1.0, 1)
        assert el[0] == eb
        n_esc = 0
        for x in vals:
            for p in vals:
                code, r = oracle.quantize(x, p, el[0], inv2[0], twoe[0])
                if code == 0:
                    assert r.tobytes() == x.tobytes()
                    n_esc += 1
                    continue
                q = code - oracle.RADIUS
                assert _exact_ok(x, r, el[0])
                ratio = (Fraction(float(x)) - Fraction(float(p))) / (2 * Fraction(float(el[0])))
                assert abs(Fraction(q) - ratio) <= Fraction(1, 2) + Fraction(1, 10 ** 5)
        assert n_esc < len(vals) ** 2


def test_quantizer_escapes_out_of_range(oracle):
    el, inv2, twoe = oracle.level_params(1e-3, 1.0, 1.0, 1)
    code, r = oracle.quantize(np.float32(100.0), np.float32(0.0), el[0], inv2[0], twoe[0])
    assert code == 0 and r == np.float32(100.0)  # |q| would exceed the radius
    code, r = oracle.quantize(np.float32(1.0), np.float32(np.nan), el[0], inv2[0], twoe[0])
    assert code == 0 and r == np.float32(1.0)


def test_level_error_bounds_eq15(oracle):
    """Eq. 15 closed forms: e_l = e / min(alpha^(l-1), beta)."""
    e = 0.5
    el, _, twoe = oracle.level_params(e, 1.0, 1.0, 5)
    assert list(el) == [0.5] * 5
    el, _, _ = oracle.level_params(e, 2.0, 8.0, 6)
    assert list(el) == [0.5, 0.25, 0.125, 0.0625, 0.0625, 0.0625]
    el, _, _ = oracle.level_params(e, 4.0, 1.0, 4)
    assert list(el) == [0.5] * 4
    el, _, twoe = oracle.level_params(e, 1.5, 2.0, 4)
    assert list(el) == [0.5, np.float32(1 / 3), 0.25, 0.25]
    assert list(twoe) == [2 * v for v in el]


def _heap_cost(freq):
    h = [f for f in freq if f > 0]
    if len(h) <= 1:
        return 0
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a = heapq.heappop(h)
        b = heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def test_huffman_optimal_kraft_prefix(oracle):
    rng = np.random.default_rng(7)
    for trial in range(400):
        n = int(rng.integers(2, 9)) if trial < 300 else int(rng.integers(9, 300))
        freq = rng.integers(0, 50 if trial % 3 else 3, size=n).astype(np.uint64)
        if trial % 5 == 0:
            freq = (2 ** rng.integers(0, 20, size=n)).astype(np.uint64)
        if np.count_nonzero(freq) < 2:
            freq[:2] = [1, 1]
        lens = oracle.huffman_lengths(freq)
        used = freq > 0
        assert np.all((lens > 0) == used)
        kraft = sum(Fraction(1, 2 ** int(l)) for l in lens[used])
        assert kraft == 1
        assert int(np.sum(freq.astype(object) * lens.astype(object))) == _heap_cost(
            [int(f) for f in freq])
        codes = oracle.canonical_codes(lens)
        words = [format(int(codes[i]), "0%db" % lens[i]) for i in range(n) if used[i]]
        for a, b in itertools.permutations(words, 2):
            assert not b.startswith(a)


def test_huffman_single_and_fibonacci(oracle):
    lens = oracle.huffman_lengths(np.array([0, 5, 0], np.uint64))
    assert list(lens) == [0, 0, 0]  # a lone symbol gets the empty code
    fib = [1, 1]
    while len(fib) < 30:
        fib.append(fib[-1] + fib[-2])
    lens = oracle.huffman_lengths(np.array(fib, np.uint64))
    assert int(lens.max()) == len(fib) - 1  # the Fibonacci worst case


def test_canonical_codes_rfc1951_example(oracle):
    rows = [l for l in open(os.path.join(GOLDEN, "rfc1951_canonical.txt"))
            if l.strip() and not l.startswith("#")]
    lens = np.array([int(r.split("|")[1]) for r in rows], np.uint8)
    want = [r.split("|")[2].strip() for r in rows]
    codes = oracle.canonical_codes(lens)
    got = [format(int(c), "0%db" % l) for c, l in zip(codes, lens)]
    assert got == want


def _linear_field(shape, seed):
    rng = np.random.default_rng(seed)
    coef = rng.integers(-3, 4, size=len(shape))
    grids = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    f = sum(c * g for c, g in zip(coef, grids)) + int(rng.integers(-5, 5))
    return f.astype(np.float32)


@pytest.mark.parametrize("interp", [0, 1, 2])
@pytest.mark.parametrize("paradigm", [0, 1])
@pytest.mark.parametrize("same", [0, 1])
def test_linear_fields_give_zero_codes(oracle, interp, paradigm, same):
    """Every stencil except the copy fallback reproduces linear functions,
    so on grids ending on an anchor every code is the zero-error code."""
    for shape, A in (((65,), 64), ((17, 33), 16), ((9, 17, 33), 8)):
        x = _linear_field(shape, seed=len(shape) + interp)
        cfg = oracle.make_config(len(shape), anchor_stride=A, interp=interp,
                                 paradigm=paradigm, same_level=same)
        _, st, codes, _ = oracle.compress(x, 0.25, oracle.EB_ABS, cfg,
                                          want_codes=True)
        assert st.bad_reads == 0 and st.double_visits == 0
        assert np.all(codes == oracle.RADIUS), (shape, interp, paradigm, same)


def test_cubic_fields_exact_where_four_knots(oracle):
    """Eq. 4 and Eq. 10 are Lagrange cubics: on a cubic polynomial every
    point predicted with all of their knots present has a zero error."""
    n, A = 65, 64
    c = np.arange(n, dtype=np.int64)
    f = (2 * c ** 3 - 3 * c ** 2 + 5 * c - 7).astype(np.float32)
    for same in (0, 1):
        cfg = oracle.make_config(1, anchor_stride=A, interp=oracle.CUBIC_NAK,
                                 same_level=same)
        _, st, codes, _ = oracle.compress(f, 0.25, oracle.EB_ABS, cfg,
                                          want_codes=True)
        for l in range(1, 7):
            s = 1 << (l - 1)
            for pos in range(s, n, 2 * s):
                if pos - 3 * s >= 0 and pos + 3 * s <= n - 1:
                    assert codes[pos] == oracle.RADIUS, (same, s, pos)
        # and the natural spline does not reproduce cubics (it is not exact)
    cfg = oracle.make_config(1, anchor_stride=A, interp=oracle.CUBIC_NAT)
    _, _, codes, _ = oracle.compress(f, 0.25, oracle.EB_ABS, cfg, want_codes=True)
    assert np.any(codes != oracle.RADIUS)


CONFIGS = [
    dict(interp=1, paradigm=0, same_level=0),
    dict(interp=0, paradigm=0, same_level=0),
    dict(interp=2, paradigm=0, same_level=1),
    dict(interp=1, paradigm=1, same_level=1),
    dict(interp=2, paradigm=1, same_level=0),
]


def test_bruteforce_tiny_1d_roundtrip(oracle):
    """All 1D integer fields of length 5 over {-2..2}, several configs: the
    decompressed field equals the compress-time reconstruction bit for bit
    and every point is within the bound."""
    for cfgd in CONFIGS:
        cfg = oracle.make_config(1, anchor_stride=4, **cfgd)
        for vals in itertools.product(range(-2, 3), repeat=5):
            x = np.array(vals, np.float32)
            s, st, _, recon = oracle.compress(x, 0.4, oracle.EB_ABS, cfg,
                                              want_recon=True)
            y = oracle.decompress(s)
            assert y.tobytes() == recon.tobytes()
            assert np.all(np.abs(y - x) <= np.float32(0.4))


@pytest.mark.parametrize("cfgd", CONFIGS)
def test_random_small_fields_roundtrip_and_coverage(oracle, cfgd):
    rng = np.random.default_rng(11)
    shapes = [(1,), (2,), (7,), (130,), (5, 5), (1, 9), (33, 17), (3, 4, 5),
              (9, 9, 9), (17, 5, 33), (1, 1, 40)]
    for shape in shapes:
        for A in (2, 4, 8, 32):
            x = (rng.standard_normal(shape).cumsum(axis=-1)).astype(np.float32)
            cfg = oracle.make_config(len(shape), anchor_stride=A, **cfgd)
            for mode, eb in ((oracle.EB_REL, 1e-2), (oracle.EB_ABS, 0.05)):
                s, st, codes, recon = oracle.compress(x, eb, mode, cfg,
                                                      want_codes=True,
                                                      want_recon=True)
                if x.max() == x.min() and mode == oracle.EB_REL:
                    continue
                assert st.bad_reads == 0 and st.double_visits == 0
                assert st.predicted + st.n_anchors == x.size
                y = oracle.decompress(s)
                assert y.tobytes() == recon.tobytes()
                e = np.float32(st.e)
                assert np.all(np.abs(y.astype(np.float64) - x) <= e)
                assert st.n_outliers == int(np.count_nonzero(codes == 0))


def test_frozen_dim_and_md_weights(oracle):
    rng = np.random.default_rng(3)
    x = rng.standard_normal((6, 33, 40)).cumsum(axis=2).cumsum(axis=1).astype(np.float32)
    for frozen in (0, 1, 2):
        for par in (0, 1):
            cfg = oracle.make_config(3, anchor_stride=8, frozen_dim=frozen,
                                     paradigm=par, md_inv_var=(1.0, 4.0, 0.5))
            s, st, codes, recon = oracle.compress(x, 1e-3, oracle.EB_REL, cfg,
                                                  want_codes=True, want_recon=True)
            assert st.bad_reads == 0 and st.predicted + st.n_anchors == x.size
            assert oracle.decompress(s).tobytes() == recon.tobytes()
            # anchors: stride 1 along the frozen dim, A along the others
            na = 1
            for d, n in enumerate(x.shape):
                na *= n if d == frozen else -(-n // 8)
            assert st.n_anchors == na
    # Eq. 14: weights proportional to 1/sigma^2 and summing to one
    iv = (1.0, 4.0, 0.5)
    for mask in range(1, 8):
        ws = [float(oracle.md_weight(iv, mask, d)) for d in range(3) if mask >> d & 1]
        tot = sum(iv[d] for d in range(3) if mask >> d & 1)
        np.testing.assert_allclose(ws, [iv[d] / tot for d in range(3) if mask >> d & 1],
                                   rtol=1e-7)
        assert abs(sum(ws) - 1.0) < 1e-6


def test_blockwise_map_roundtrip(oracle):
    rng = np.random.default_rng(5)
    x = rng.standard_normal((40, 70)).cumsum(0).cumsum(1).astype(np.float32)
    nb = (-(-40 // 32)) * (-(-70 // 32))
    bm = rng.integers(0, 8, size=nb).astype(np.uint8)
    bm[(bm & 3) == 3] = 1
    cfg = oracle.make_config(2, anchor_stride=16, blockmap=bm)
    s, st, _, recon = oracle.compress(x, 1e-3, oracle.EB_REL, cfg, want_recon=True)
    assert st.bad_reads == 0 and st.predicted + st.n_anchors == x.size
    assert oracle.decompress(s).tobytes() == recon.tobytes()


def test_relative_bound_and_constant_field(oracle):
    x = np.linspace(-3, 5, 1000, dtype=np.float32).reshape(10, 100)
    _, st, _, _ = oracle.compress(x, 1e-3, oracle.EB_REL)
    assert st.e == np.float32(1e-3 * (float(x.max()) - float(x.min())))
    c = np.full((7, 9), 2.5, np.float32)
    s, _, _, _ = oracle.compress(c, 1e-3, oracle.EB_REL)
    assert len(s) == 512
    assert np.array_equal(oracle.decompress(s), c)
    with pytest.raises(oracle.OracleError):
        oracle.compress(np.array([1.0, np.nan], np.float32), 1e-3, oracle.EB_REL)


def test_corrupt_streams_rejected(oracle):
    x = np.random.default_rng(1).standard_normal((20, 30)).astype(np.float32)
    s, _, _, _ = oracle.compress(x, 1e-2)
    with pytest.raises(oracle.OracleError):
        oracle.decompress(s[:400])
    bad = bytearray(s)
    bad[0] ^= 0xFF
    with pytest.raises(oracle.OracleError):
        oracle.decompress(bytes(bad))
    # flip the first bit of lane 1 of chunk 0: the code of point 1 (never an
    # anchor) changes, so the decoder must either reject the stream (the
    # lane no longer ends on its stored bit count, or the escape count no
    # longer matches) or return a different field
    hdr = np.frombuffer(s[:512], np.uint8)
    ocw = int(hdr[264:272].view(np.uint64)[0])
    obits = int(hdr[288:296].view(np.uint64)[0])
    lane0_bits = int(np.frombuffer(s[ocw:ocw + 2], np.uint16)[0])
    assert int(np.frombuffer(s[ocw + 2:ocw + 4], np.uint16)[0]) > 0
    word = obits + 4 * (lane0_bits // 32)
    bit = 31 - lane0_bits % 32
    bad = bytearray(s)
    w = int.from_bytes(bad[word:word + 4], "little") ^ (1 << bit)
    bad[word:word + 4] = w.to_bytes(4, "little")
    try:
        y = oracle.decompress(bytes(bad))
    except oracle.OracleError:
        return
    assert not np.array_equal(y, oracle.decompress(s))


def test_error_bound_on_workload_fields(oracle):
    from paper_2311_12133_gb300 import fields as F
    for kind, shape in (("bumps", (48, 40, 36)), ("grf", (40, 40, 40)),
                        ("lognormal", (32, 32, 32)), ("climate2d", (90, 180))):
        x = F.make(kind, shape, 3)
        for eps in (1e-2, 1e-3, 1e-4):
            s, st, _, recon = oracle.compress(x, eps, oracle.EB_REL, want_recon=True)
            y = oracle.decompress(s)
            assert y.tobytes() == recon.tobytes()
            assert np.all(np.abs(y.astype(np.float64) - x) <= st.e)
