"""Pins of the oracle's auto-tuner (Sec. 6) against closed forms, brute
force over the candidate lists and the optimal-prefix-code cost.

Every expected value here is computed independently of the oracle's tuner:
finite differences with numpy, a heap-based Huffman cost, lattice sampling
restated from the rule it follows, and argmins taken in Python over
compression tests of the (separately pinned) level sweep.
"""
from __future__ import annotations

import heapq
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_12133_gb300 import fields

ALPHAS = (1.0, 1.25, 1.5, 1.75, 2.0)
BETAS = (2.0, 4.0, 8.0, 16.0)
BLOCK_CODES = (0, 1, 5, 2, 6)


def optimal_code_bits(hist) -> int:
    """Total length of an optimal prefix code: the sum of the weights of the
    internal nodes of any Huffman tree (independent of tie-breaking).  A
    lone symbol costs nothing (it gets the empty code)."""
    w = [int(v) for v in np.asarray(hist).ravel() if v]
    if len(w) <= 1:
        return 0
    heapq.heapify(w)
    total = 0
    while len(w) > 1:
        a = heapq.heappop(w)
        b = heapq.heappop(w)
        total += a + b
        heapq.heappush(w, a + b)
    return total


def lattice_stride(ndim: int, rate: float) -> int:
    t = 1
    while t ** ndim * rate < 1.0:
        t += 1
    return t


def sample_block_slices(shape, A: int, rate: float):
    """Blocks of A+1 points every tau blocks per dim, tau the smallest
    stride with at most floor(rate*N/A^ndim + 0.5) (>= 1) blocks."""
    ndim = len(shape)
    nb = [(n - 1) // A for n in shape]
    N = int(np.prod(shape))
    target = max(1, int(math.floor(rate * N / A ** ndim + 0.5)))
    tau = 1
    while np.prod([-(-max(m, 1) // tau) for m in nb]) > target:
        tau += 1
    per_dim = []
    for d in range(ndim):
        if nb[d]:
            per_dim.append([slice(j * tau * A, j * tau * A + A + 1)
                            for j in range(-(-nb[d] // tau))])
        else:
            per_dim.append([slice(0, shape[d])])
    return [tuple(s) for s in itertools.product(*per_dim)]


def quiet_params(**kw):
    base = dict(tune_levels=0, tune_eb=0, tune_freeze=0, tune_lorenzo=0,
                tune_blockwise=0)
    base.update(kw)
    return O.default_tune_params(**base)


# ------------------------------------------------------------ candidates
def test_candidate_lists():
    """Sec. 6.2: linear x (orders + MD), then not-a-knot and natural cubic
    x (orders + MD) x same-level off/on.  3D: 7 + 14 + 14 = 35."""
    def count(ndim, frozen=-1, **kw):
        tp = O.default_tune_params(**kw)
        j = 0
        while O.tune_candidate(ndim, frozen, j, tp) is not None:
            j += 1
        return j

    assert count(3) == 35
    assert count(2) == 15
    assert count(1) == 5
    assert count(3, frozen=1) == 15
    assert count(3, allow_natural=0) == 21
    assert count(3, allow_same_level=0) == 21
    # 1D-style orders in lexicographic order, then MD, for every kind
    perms = list(itertools.permutations(range(3)))
    for j, p in enumerate(perms):
        assert O.tune_candidate(3, -1, j) == (O.LINEAR, O.P1D, p, 0)
    assert O.tune_candidate(3, -1, 6)[:2] == (O.LINEAR, O.PMD)
    assert O.tune_candidate(3, -1, 7) == (O.CUBIC_NAK, O.P1D, (0, 1, 2), 0)
    assert O.tune_candidate(3, -1, 8) == (O.CUBIC_NAK, O.P1D, (0, 1, 2), 1)
    assert O.tune_candidate(3, -1, 21) == (O.CUBIC_NAT, O.P1D, (0, 1, 2), 0)
    # the frozen dim never appears in an order
    for j in range(15):
        k, par, order, same = O.tune_candidate(3, 1, j)
        assert 1 not in order[:2] and order[2] == 255


# ----------------------------------------------------------------- stats
def test_stats_quartic_closed_form():
    """Sec. 6.1 on x = j^4 (dim 1 only): cubic (not-a-knot) interpolation
    of a quartic misses by 4!/24 * (-3)(-1)(1)(3) = 9 everywhere; linear
    misses by 6 j^2 + 1; dims 0 and 2 are exact."""
    n = 20
    j = np.arange(n, dtype=np.float64)
    x = np.broadcast_to((j ** 4)[None, :, None], (n, n, n)).astype(np.float32)
    rate = 0.002
    t = lattice_stride(3, rate)
    assert t == 8
    pts = np.arange(3, n - 3, t)
    cnt = len(pts) ** 3
    cfg, rep = O.tune(x, 1.0, O.EB_ABS, quiet_params(sample_rate=rate))
    assert rep.stats_count == cnt
    sq = lambda err: math.floor(min(abs(err), 65536.0) ** 2 * 256.0)
    lin1 = sum(sq(6 * jj * jj + 1) for jj in pts) * len(pts) ** 2
    assert list(rep.mse_cub) == [0, cnt * sq(9), 0]
    assert list(rep.mse_lin) == [0, lin1, 0]
    assert rep.nonsmooth_dim == 1
    # Eq. 14 weights from 1/sigma^2: count * 256 / max(sum, 1)
    assert cfg.md_inv_var[0] == cnt * 256.0
    assert cfg.md_inv_var[1] == cnt * 256.0 / (cnt * sq(9))
    assert cfg.md_inv_var[2] == cnt * 256.0


def test_stats_2d_lattice_and_small_fields():
    x = fields.make("grf", (50, 41), seed=4)
    t = lattice_stride(2, 0.002)
    assert t == 23
    _, rep = O.tune(x, 1e-3, O.EB_REL, quiet_params())
    assert rep.stats_count == len(range(3, 47, t)) * len(range(3, 38, t))
    # a dim shorter than 7 leaves no lattice point: equal weights
    cfg, rep = O.tune(fields.make("grf", (6, 40), seed=4), 1e-3, O.EB_REL,
                      quiet_params())
    assert rep.stats_count == 0 and rep.nonsmooth_dim == -1
    assert list(cfg.md_inv_var) == [1.0, 1.0, 1.0]


# --------------------------------------------------------------- Lorenzo
@pytest.mark.parametrize("shape,A", [((129,), 128), ((33, 33), 32),
                                     ((9, 9, 9), 8), ((33, 33, 33), 32)])
def test_lorenzo_bits_finite_differences(shape, A):
    """Sec. 6.5: on integer data with e = 1/2 every prediction is exact in
    binary32 and q = x - p, so order-1 (order-2) Lorenzo codes are the
    first (second) finite differences along every dim with zero padding."""
    rng = np.random.default_rng(7)
    x = rng.integers(0, 21, size=shape).astype(np.float32)
    _, rep = O.tune(x, 0.5, O.EB_ABS,
                    quiet_params(tune_lorenzo=1, anchor_stride=A))
    assert rep.n_sample_blocks == 1
    for order in (1, 2):
        d = x.astype(np.int64)
        for ax in range(len(shape)):
            for _ in range(order):
                d = np.diff(d, axis=ax, prepend=0)
        _, counts = np.unique(d, return_counts=True)
        assert rep.lorenzo_bits[order - 1] == optimal_code_bits(counts), order


# ------------------------------------------------- global tuning (6.2, 6.4)
def brute_force_global(x, e, A, rate, frozen, md_inv_var):
    """Per-level argmin (first index on ties) of the summed level scores
    over the sample blocks, coarsest level first, each level tested with
    the levels above it already fixed; then the (alpha, beta) grid by
    estimated bits."""
    ndim = x.ndim
    blocks = [np.ascontiguousarray(x[s]) for s in
              sample_block_slices(x.shape, A, rate)]
    order = [d for d in range(ndim) if d != frozen]
    cfg = O.make_config(ndim, anchor_stride=A, frozen_dim=frozen,
                        md_inv_var=md_inv_var, order=order)
    L = int(math.log2(A))
    choice = {}
    for l in range(L, 0, -1):
        scores = []
        j = 0
        while (cand := O.tune_candidate(ndim, frozen, j)) is not None:
            kind, par, od, same = cand
            cfg.interp[l - 1], cfg.paradigm[l - 1] = kind, par
            cfg.same_level[l - 1] = same
            for q in range(3):
                cfg.order[l - 1][q] = od[q]
            scores.append(sum(int(O.subfield_test(b, cfg, e, l)[0][l - 1])
                              for b in blocks))
            j += 1
        best = int(np.argmin(scores))
        choice[l] = (best, scores[best])
        kind, par, od, same = O.tune_candidate(ndim, frozen, best)
        cfg.interp[l - 1], cfg.paradigm[l - 1] = kind, par
        cfg.same_level[l - 1] = same
        for q in range(3):
            cfg.order[l - 1][q] = od[q]

    def bits(c):
        hist = np.zeros(65536, np.uint64)
        nout = na = 0
        for b in blocks:
            _, h, no, a = O.subfield_test(b, c, e, 1)
            hist += h
            nout += no
            na += a
        return optimal_code_bits(hist) + 32 * nout + 32 * na

    grid = [(1.0, 1.0)] + [(a, b) for a in ALPHAS[1:] for b in BETAS]
    best_bits, best_ab = None, None
    for a, b in grid:
        cfg.alpha, cfg.beta = a, b
        v = bits(cfg)
        if best_bits is None or v < best_bits:
            best_bits, best_ab = v, (a, b)
    cfg.alpha, cfg.beta = best_ab
    return cfg, choice, bits(cfg), len(blocks)


@pytest.mark.parametrize("kind,shape,A,rate,eb", [
    ("grf", (65, 65), 64, 0.01, 1e-3),
    ("bumps", (40, 40, 40), 8, 0.1, 1e-3),
    ("grf", (33, 48, 30), 16, 0.05, 1e-2),
])
def test_global_tuning_is_brute_force_argmin(kind, shape, A, rate, eb):
    x = fields.make(kind, shape, seed=11)
    tp = O.default_tune_params(block_rate=rate, anchor_stride=A,
                               tune_freeze=0, tune_lorenzo=0,
                               tune_blockwise=0)
    cfg, rep = O.tune(x, eb, O.EB_REL, tp)
    e = np.float32(eb * (float(x.max()) - float(x.min())))
    ref, choice, bits, nblk = brute_force_global(
        x, float(e), A, rate, -1, list(cfg.md_inv_var))
    assert rep.n_sample_blocks == nblk
    L = int(math.log2(A))
    for l in range(1, L + 1):
        assert rep.level_choice[0][l - 1] == choice[l][0], l
        assert rep.level_score[0][l - 1] == choice[l][1], l
        assert cfg.interp[l - 1] == ref.interp[l - 1]
        assert cfg.paradigm[l - 1] == ref.paradigm[l - 1]
        assert cfg.same_level[l - 1] == ref.same_level[l - 1]
        assert list(cfg.order[l - 1]) == list(ref.order[l - 1])
    assert (cfg.alpha, cfg.beta) == (ref.alpha, ref.beta)
    assert rep.bits[0] == bits


def test_tuned_config_round_trips_within_bound():
    x = fields.make("grf", (48, 40, 36), seed=2)
    cfg, _ = O.tune(x, 1e-3)
    stream, st, _, _ = O.compress(x, 1e-3, config=cfg)
    y = O.decompress(stream)
    assert np.all(np.abs(y.astype(np.float64) - x) <= st.e)
    default, _, _, _ = O.compress(x, 1e-3)
    assert len(stream) <= len(default) * 1.02


# -------------------------------------------------------- freezing (6.3)
def test_freeze_choice_follows_estimates():
    x = fields.make("grf", (40, 36, 33), seed=5)
    tp = O.default_tune_params(tune_blockwise=0, tune_lorenzo=0,
                               anchor_stride=8, block_rate=0.1)
    cfg, rep = O.tune(x, 1e-3, O.EB_REL, tp)
    assert rep.froze == int(rep.bits[1] < rep.bits[0])
    assert cfg.frozen_dim == (rep.nonsmooth_dim if rep.froze else -1)


def test_freeze_picks_the_rough_dimension():
    """Smooth in-plane, white noise across planes: the statistics name the
    noisy dim, and interpolating only within planes wins (Sec. 6.3)."""
    rng = np.random.default_rng(3)
    n = 40
    j = np.linspace(0, 2 * np.pi, n)
    plane = np.sin(j)[:, None] * np.cos(j)[None, :]
    x = (plane[None, :, :] * (1 + rng.normal(0, 1, (n, 1, 1)))
         + rng.normal(0, 1, (n, 1, 1))).astype(np.float32)
    tp = O.default_tune_params(tune_blockwise=0, tune_lorenzo=0,
                               anchor_stride=8, block_rate=0.1)
    cfg, rep = O.tune(x, 1e-3, O.EB_REL, tp)
    assert rep.nonsmooth_dim == 0
    assert rep.froze == 1 and cfg.frozen_dim == 0
    assert rep.bits[1] < rep.bits[0]


# ------------------------------------------------------ block-wise (6.6)
def sub_blocks(shape, bs, sub_frac, frozen):
    ndim = len(shape)
    Q = max(5, int(math.floor(bs / 32 * 32 * sub_frac ** (1 / ndim) + 0.5)))
    nb = [-(-n // bs) for n in shape]
    out = []
    for idx in itertools.product(*[range(m) for m in nb]):
        sl, qmin = [], None
        for d in range(ndim):
            b0 = idx[d] * bs
            ext = min(bs, shape[d] - b0)
            q = min(ext, Q)
            s0 = b0 + (ext - q) // 2
            sl.append(slice(s0, s0 + q))
            if d != frozen:
                qmin = q if qmin is None else min(qmin, q)
        As = 2
        while As * 2 <= max(qmin - 1, 1):
            As *= 2
        out.append((tuple(sl), As))
    return Q, out


def test_blockwise_is_brute_force_argmin():
    x = fields.make("bumps", (70, 64, 40), seed=9)
    tp = O.default_tune_params(tune_freeze=0, tune_lorenzo=0,
                               tune_levels=0, tune_eb=0)
    cfg, rep = O.tune(x, 1e-3, O.EB_REL, tp)
    e = float(np.float32(1e-3 * (float(x.max()) - float(x.min()))))
    Q, blocks = sub_blocks(x.shape, 32, 0.04, cfg.frozen_dim)
    assert Q == 11
    bm = cfg._blockmap_ref
    assert cfg.blockwise == 1 and bm.size == len(blocks) == 3 * 2 * 2
    for b, (sl, As) in enumerate(blocks):
        xs = np.ascontiguousarray(x[sl])
        best, bj = None, None
        for code in BLOCK_CODES:
            c = O.make_config(3, anchor_stride=As, interp=code & 3,
                              same_level=code >> 2)
            tot = int(O.subfield_test(xs, c, e, 1)[0].sum())
            if best is None or tot < best:
                best, bj = tot, code
        assert bm[b] == bj, b


def test_blockwise_semantics():
    """Blocks holding a plane (every candidate exact) keep the first code
    (linear); blocks holding a cubic polynomial take a cubic spline."""
    n = 64
    i, j, k = np.meshgrid(*[np.arange(n, dtype=np.float64)] * 3,
                          indexing="ij")
    lin = i + 2 * j + 3 * k
    cub = ((i / 8) ** 3 + (j / 8) ** 3 + (k / 8) ** 3) * 10
    x = np.where(i < 32, lin, cub).astype(np.float32)
    tp = O.default_tune_params(tune_freeze=0, tune_lorenzo=0,
                               tune_levels=0, tune_eb=0)
    cfg, _ = O.tune(x, 1e-4, O.EB_ABS, tp)
    bm = cfg._blockmap_ref.reshape(2, 2, 2)
    assert np.all(bm[0] == 0)
    assert np.all(np.isin(bm[1], (1, 5)))


def test_tune_argument_errors():
    x = fields.make("grf", (20, 20), seed=1)
    with pytest.raises(O.OracleError):
        O.tune(x, 0.0)
    with pytest.raises(O.OracleError):
        O.tune(x, 1e-3, 7)
    with pytest.raises(O.OracleError):
        O.tune(x, 1e-3, O.EB_REL, O.default_tune_params(block_size=0))
    # a constant field has nothing to tune: defaults, no block map
    cfg, rep = O.tune(np.ones((20, 20), np.float32), 1e-3)
    assert cfg.blockwise == 0 and cfg.anchor_stride == 64
