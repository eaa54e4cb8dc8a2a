"""The tuner's compression-test score (Sec. 6.2), restated from scratch.

The score of a candidate at level l is the sum, over the points level l
predicts, of floor(min(|x - p| * r_l, 2^24 - 1) * 256) in binary32, where p
is the candidate's prediction from the reconstructed coarser points and
r_l = (float)(1 / e_l).  This file re-derives every ingredient without the
oracle's sweep, which it then checks:

- the points of a level come from the hierarchy's parities (Sec. 5.1): the
  new points at stride s are on the stride-s grid and off the stride-2s
  grid; a 1D-style pass along pi_j takes those odd on pi_j, on the stride-s
  grid on the earlier directions and on the stride-2s grid on the later
  ones; a multi-dimensional sub-pass k' those with exactly k' odd
  coordinates (Eq. 8);
- stencil weights are those of cubic-spline interpolation through the
  knots that exist (scipy CubicSpline, not-a-knot or natural, as in Eq. 4
  and Eq. 6), the midpoint rule of Eq. 2, and linear extrapolation through
  the two left knots where no right knot exists;
- the linear quantizer in exact rational arithmetic: q is the integer
  nearest (x - p) / 2e, accepted iff |p + 2eq - x| <= e (else the point
  keeps x); exactly halfway, where both neighbours meet the bound, the
  binary32 reading of the quantizer decides.

Inputs are small integers and e = 49/32, so every prediction of the linear
and not-a-knot stencils is a dyadic rational of few bits: its exact value is
what any order of binary32 operations gives.  Where that holds (asserted
per level, not assumed) the scores must match exactly; elsewhere (the
1/40 of Eq. 6 below the coarsest level, 1/3 weights) within a relative
1e-4, and the mutants at the end show that the plausible mistakes move a
score by far more than that.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O

E = Fraction(49, 32)
LIN, NAK, NAT = 0, 1, 2
P1D, PMD = 0, 1


def spline_weights(knots, bc):
    from scipy.interpolate import CubicSpline
    out = []
    for j in range(len(knots)):
        y = np.zeros(len(knots))
        y[j] = 1.0
        w = float(CubicSpline(np.array(knots, float), y, bc_type=bc)(0.0))
        out.append(Fraction(w).limit_denominator(4096))
    return out


_WEIGHTS = {}


def weights(kind, knots):
    key = (kind, tuple(knots))
    if key not in _WEIGHTS:
        _WEIGHTS[key] = spline_weights(knots, "not-a-knot" if kind == NAK else "natural")
    return _WEIGHTS[key]


def is_f32(v: Fraction) -> bool:
    return Fraction(float(np.float32(float(v)))) == v


class Sweep:
    """Levels L..l_stop of one candidate configuration on a small field."""

    def __init__(self, x, A, levels, el_scale=1, mutant=None, iv=(1.0, 1.0, 1.0)):
        self.x = x
        self.iv = iv
        self.shape = x.shape
        self.A = A
        self.L = int(math.log2(A))
        self.levels = levels  # l -> (kind, paradigm, order)
        self.mutant = mutant
        self.el_scale = el_scale
        self.R = {}
        for c in itertools.product(*[range(n) for n in self.shape]):
            if all(v % A == 0 for v in c):
                self.R[c] = Fraction(int(x[c]))
        self.exact = {}
        self.ties = 0

    def nb(self, c, d, o, s):
        cc = list(c)
        cc[d] += o * s
        if not 0 <= cc[d] < self.shape[d]:
            return None
        return self.R[tuple(cc)]

    def predict_dim(self, kind, c, d, s):
        m1, p1 = self.nb(c, d, -1, s), self.nb(c, d, 1, s)
        m3, p3 = self.nb(c, d, -3, s), self.nb(c, d, 3, s)
        if p1 is None:
            return m1 + (m1 - m3) / 2 if m3 is not None else m1
        if kind == LIN or (m3 is None and p3 is None):
            return (m1 + p1) / 2
        pairs = [(k, v) for k, v in ((-3, m3), (-1, m1), (1, p1), (3, p3)) if v is not None]
        w = weights(kind, [k for k, _ in pairs])
        return sum(wk * v for wk, (_, v) in zip(w, pairs))

    def points(self, l, par, order, j):
        s = 1 << (l - 1)
        nd = len(self.shape)
        out = []
        for c in itertools.product(*[range(n) for n in self.shape]):
            if any(v % s for v in c):
                continue
            odd = [d for d in range(nd) if (c[d] // s) % 2 == 1]
            if par == P1D:
                if c[order[j]] % (2 * s) != s:
                    continue
                if any(c[order[m]] % (2 * s) for m in range(j + 1, nd)):
                    continue
            elif len(odd) != j + 1:
                continue
            out.append((c, odd))
        return out

    def run(self, l_stop=1):
        nd = len(self.shape)
        scores = {}
        for l in range(self.L, l_stop - 1, -1):
            kind, par, order = self.levels[l]
            s = 1 << (l - 1)
            el = E / self.el_scale
            r_l = np.float32(1.0 / float(el))
            exact = True
            total = 0
            for j in range(nd):
                new = {}
                for c, odd in self.points(l, par, order, j):
                    if par == P1D:
                        p = self.predict_dim(kind, c, order[j], s)
                    else:
                        # Eq. 8: the 1D predictions along the odd
                        # directions, ascending, weighted by Eq. 14's
                        # inverse variances normalised over those
                        # directions (the sum in double, each weight
                        # rounded once), accumulated in binary32
                        tot = 0.0
                        for dd in odd:
                            tot += float(self.iv[dd])
                        acc, p_ex = None, Fraction(0)
                        for dd in odd:
                            w = np.float32(float(self.iv[dd]) / tot)
                            pd = self.predict_dim(kind, c, dd, s)
                            if not is_f32(pd):
                                exact = False
                            t = np.float32(w * np.float32(float(pd)))
                            acc = t if acc is None else np.float32(acc + t)
                            p_ex += Fraction(float(w)) * pd
                        p = Fraction(float(acc))
                        if p != p_ex:
                            exact = False
                    if not is_f32(p):
                        exact = False
                        p = Fraction(float(np.float32(float(p))))
                    xv = Fraction(int(self.x[c]))
                    d = xv - p
                    if not is_f32(d):
                        exact = False
                    # the score, in binary32 as defined
                    v = np.float32(abs(float(np.float32(float(d))))) * r_l
                    v = min(v, np.float32(16777215.0))
                    total += int(math.floor(float(v * np.float32(256.0))))
                    # quantize against e_l in exact arithmetic
                    t = abs(d) / (2 * el)
                    k = math.floor(t + Fraction(1, 2))
                    if (t + Fraction(1, 2)).denominator == 1:
                        # halfway: both neighbours meet the bound, and the
                        # paper fixes no choice; take the binary32 reading
                        # |d| * (1/2e) + 1/2, truncated
                        self.ties += 1
                        inv2 = np.float32(1.0 / (2.0 * float(el)))
                        k = int(np.float32(np.float32(abs(float(d))) * inv2) + np.float32(0.5))
                    q = k * (1 if d >= 0 else -1)
                    rec = p + 2 * el * q
                    new[c] = rec if abs(q) < 32768 and abs(rec - xv) <= el else xv
                if self.mutant == "score_known" and j == 0:
                    # a plausible mistake: also score the stride-2s points
                    for c in itertools.product(*[range(0, n, 2 * s) for n in self.shape]):
                        if c in self.R and not all(v % self.A == 0 for v in c):
                            total += 256
                self.R.update(new)
            scores[l] = total
            self.exact[l] = exact
        return scores


def int_field(shape, seed):
    rng = np.random.default_rng(seed)
    g = np.meshgrid(*[np.linspace(0, 2.5, n) for n in shape], indexing="ij")
    base = 20 * np.sin(sum((i + 1) * a for i, a in enumerate(g)))
    return np.rint(base + rng.integers(-4, 5, size=shape)).astype(np.float32)


def oracle_scores(x, A, levels):
    nd = x.ndim
    cfg = O.make_config(nd, anchor_stride=A,
                        interp=[levels[l][0] for l in sorted(levels)],
                        paradigm=[levels[l][1] for l in sorted(levels)],
                        order=[list(levels[l][2]) for l in sorted(levels)])
    sc, _, _, _ = O.subfield_test(x, cfg, float(E), 1)
    return {l: int(sc[l - 1]) for l in levels}


CASES = [
    ((33,), 16, [(LIN, P1D), (NAK, P1D), (NAT, P1D)]),
    ((17, 13), 8, [(LIN, P1D), (NAK, P1D), (LIN, PMD), (NAK, PMD), (NAT, P1D)]),
    ((17, 13, 11), 8, [(LIN, P1D), (NAK, P1D), (LIN, PMD), (NAK, PMD)]),
]


@pytest.mark.parametrize("shape,A,kinds", CASES)
def test_subfield_scores_restated(shape, A, kinds):
    x = int_field(shape, seed=len(shape))
    nd = len(shape)
    L = int(math.log2(A))
    n_exact = 0
    for kind, par in kinds:
        for order in itertools.permutations(range(nd)):
            if par == PMD and order != tuple(range(nd)):
                continue
            levels = {l: (kind, par, order) for l in range(1, L + 1)}
            sw = Sweep(x, A, levels)
            want = sw.run()
            got = oracle_scores(x, A, levels)
            for l in range(L, 0, -1):
                if sw.exact[l] and all(sw.exact[m] for m in range(l, L + 1)):
                    assert got[l] == want[l], (kind, par, order, l)
                    n_exact += 1
                else:
                    assert got[l] == pytest.approx(want[l], rel=1e-4), (kind, par, order, l)
    assert n_exact >= len(kinds)  # the exact comparisons are not vacuous


def test_mixed_levels_restated():
    """Per-level candidates as the tuner assembles them: a different
    interpolator, paradigm and order at each level."""
    x = int_field((17, 17, 9), seed=7)
    levels = {3: (NAK, P1D, (2, 0, 1)), 2: (LIN, PMD, (0, 1, 2)), 1: (NAK, P1D, (1, 2, 0))}
    sw = Sweep(x, 8, levels)
    want = sw.run()
    got = oracle_scores(x, 8, levels)
    for l in (3, 2, 1):
        assert got[l] == pytest.approx(want[l], rel=1e-4)


def test_tuner_level_scores_restated():
    """The tuner's reported per-level choice and score on a field that is
    one sample block: each level's argmin over the candidate list (first
    index on ties), with the coarser levels fixed, from the restated
    sweep."""
    for shape, A in (((17, 17), 16), ((9, 9, 9), 8)):
        x = int_field(shape, seed=3)
        nd, L = len(shape), int(math.log2(A))
        tp = O.default_tune_params(anchor_stride=A, tune_eb=0, tune_freeze=0,
                                   tune_lorenzo=0, tune_blockwise=0,
                                   allow_natural=0, allow_same_level=0)
        cfg, rep = O.tune(x, float(E), O.EB_ABS, tp)
        assert rep.n_sample_blocks == 1
        iv = list(cfg.md_inv_var)[:nd]
        cands = []
        while (c := O.tune_candidate(nd, -1, len(cands), tp)) is not None:
            cands.append(c)
        assert len(cands) == 2 * (math.factorial(nd) + 1)
        chosen = {}
        for l in range(L, 0, -1):
            scores, exact = [], []
            for kind, par, od, _ in cands:
                levels = dict(chosen)
                for m in range(1, l + 1):
                    levels[m] = (kind, par, tuple(od[:nd]))
                sw = Sweep(x, A, levels, iv=iv)
                scores.append(sw.run(l_stop=l)[l])
                exact.append(all(sw.exact.values()))
            best = int(np.argmin(scores))
            # the argmin is determined where every score near the best is
            # exact (ties then go to the first index, as in the oracle)
            near = [j for j, v in enumerate(scores) if v <= scores[best] * (1 + 1e-4)]
            assert all(exact[j] for j in near) or len(near) == 1, "near-tie of inexact scores"
            assert rep.level_choice[0][l - 1] == best, (shape, l)
            if exact[best]:
                assert rep.level_score[0][l - 1] == scores[best], (shape, l)
            else:
                assert rep.level_score[0][l - 1] == pytest.approx(scores[best], rel=1e-4)
            kind, par, od, _ = cands[best]
            chosen[l] = (kind, par, tuple(od[:nd]))


def test_mutants_move_the_score():
    """The plausible mistakes the restatement guards against change a score
    by far more than the 1e-4 tolerance: the level bound taken at twice its
    value, the stride-2s points scored as new ones, a transposed order."""
    x = int_field((17, 13, 11), seed=3)
    levels = {l: (NAK, P1D, (0, 1, 2)) for l in (1, 2, 3)}
    base = Sweep(x, 8, levels).run()
    got = oracle_scores(x, 8, levels)
    assert got == base
    scaled = Sweep(x, 8, levels, el_scale=Fraction(1, 2)).run()
    known = Sweep(x, 8, levels, mutant="score_known").run()
    swapped = Sweep(x, 8, {l: (NAK, P1D, (1, 0, 2)) for l in (1, 2, 3)}).run()
    for m in (scaled, known, swapped):
        assert any(abs(m[l] - got[l]) > 1e-3 * got[l] for l in (1, 2, 3))
