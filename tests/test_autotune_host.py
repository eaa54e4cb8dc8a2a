"""Host logic of the level-schedule search driver (no GPU): how fields are
grouped into shape classes, how tables merge, the benchmark mix, and what
the shipped table holds for the benchmark field."""
import math

import pytest

from paper_2311_12133_gb300 import hpez


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2311_12133_gb300 import build as B
    B.build()


def test_class_of_groups_by_half_octave_and_config():
    from paper_2311_12133_gb300 import autotune
    # 362 and 363 straddle a half-octave boundary (2 log2 n = 17.0 at 362.04)
    a = autotune.class_of((362, 362, 362), None)
    b = autotune.class_of((363, 363, 363), None)
    c = autotune.class_of((370, 380, 390), None)
    assert a != b and b == c
    md = {"paradigm": 1, "interp": 0}
    assert autotune.class_of((363, 363, 363), md) != b
    assert autotune.class_of((363, 363, 363), md) == autotune.class_of((380, 370, 390), md)
    # the class is the level-1 key without stride, interpolator, paradigm
    # and direction, plus the configuration
    k = hpez.hpez_level_key_of((363, 363, 363), None, 1, False)
    assert b == (k[:4], ())


def test_merge_first_wins():
    from paper_2311_12133_gb300 import autotune
    k1 = (3, 17, 17, 17, 1, 0, 1, 0)
    k2 = (3, 17, 17, 17, 1, 0, 1, 1)
    k3 = (2, 0, 21, 23, 1, 1, 0, 0)
    t1, t2, t3 = hpez.Tuning(), hpez.Tuning(), hpez.Tuning()
    t1.set(k1, hpez.HPEZ_FAM_MD3W, chunks=24, time_us=10.0)
    t2.set(k1, hpez.HPEZ_FAM_MD3, (0, 8, 0), time_us=20.0)
    t2.set(k2, hpez.HPEZ_FAM_MD3W, chunks=12, time_us=30.0)
    t3.set(k2, hpez.HPEZ_FAM_PASS, time_us=40.0)
    t3.set(k3, hpez.HPEZ_FAM_FUSED, (1, 8, 128), time_us=50.0)
    m = autotune.merge_first_wins([t1, t2, t3])
    assert len(m) == 3
    v1, v2, v3 = m.get(k1), m.get(k2), m.get(k3)
    assert v1.family == hpez.HPEZ_FAM_MD3W and v1.chunks == 24 and v1.time_us == 10.0
    assert v2.family == hpez.HPEZ_FAM_MD3W and v2.chunks == 12 and v2.time_us == 30.0
    assert v3.astuple() == (hpez.HPEZ_FAM_FUSED, 1, 8, 128, 0)
    # the inputs are left as they were
    assert len(t1) == 1 and len(t2) == 2 and len(t3) == 2
    assert t2.get(k1).family == hpez.HPEZ_FAM_MD3


def test_mix_specs_cover_each_configuration():
    from paper_2311_12133_gb300 import autotune, fields
    mix = fields.batch_mix(64, seed=0)
    specs = autotune.mix_specs(64, seed=0)
    assert len(specs) == 2 * len(mix)
    assert [s[:4] for s in specs[:64]] == mix and [s[:4] for s in specs[64:]] == mix
    assert all(s[4] is None for s in specs[:64])
    assert all(s[4] == {"paradigm": 1, "interp": 0} for s in specs[64:])
    # sizes within the mix's bounds, about a third of the fields 2D
    npts = [math.prod(s[1]) for s in mix]
    assert min(npts) >= 8 * 8 and max(npts) <= 2 * 256 * 384 * 384
    n2 = sum(len(s[1]) == 2 for s in mix)
    assert 10 <= n2 <= 35


def test_shipped_table_holds_the_benchmark_finest_level():
    """The benchmark field's tuned predictor (linear multi-dimensional at
    every level) finds a warp-strip chunk count for its finest level; a
    decompression level without an entry of its own takes the compression
    level's, so one of the two directions must hold a warp-strip entry."""
    from paper_2311_12133_gb300 import autotune
    t = hpez.Tuning(autotune.SHIPPED)
    cfg = hpez.make_config(3, paradigm=1, interp=0)
    kc = hpez.hpez_level_key_of((512, 512, 512), cfg, 1, False)
    kd = hpez.hpez_level_key_of((512, 512, 512), cfg, 1, True)
    vc, vd = t.get(kc), t.get(kd)
    assert vc is not None, kc
    assert vc.family == hpez.HPEZ_FAM_MD3W and 1 <= vc.chunks <= 256 and vc.time_us > 0.0
    if vd is not None:
        assert vd.time_us > 0.0
