"""The level-schedule table of the batched and served forms (host logic,
no GPU): keys of a field's levels, entries, and the text file."""
import os

import pytest

from paper_2311_12133_gb300 import hpez


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2311_12133_gb300 import build as B
    B.build()


def test_level_keys():
    # (ndim, floor(2 log2 n) of each slot, stride, interp, paradigm, decomp)
    k = hpez.hpez_level_key_of((100, 500, 500), None, 1, False)
    assert k == (3, 13, 17, 17, 1, hpez.HPEZ_CUBIC_NAK, 0, 0)
    k = hpez.hpez_level_key_of((128, 128, 128), None, 3, True)
    assert k == (3, 14, 14, 14, 4, hpez.HPEZ_CUBIC_NAK, 0, 1)
    k = hpez.hpez_level_key_of((1800, 3600), None, 2, False)
    assert k == (2, 0, 21, 23, 2, hpez.HPEZ_CUBIC_NAK, 0, 0)
    # half-octaves: 335 and 512 (or 362 and 363) fall in different classes
    import math
    for n in (1, 2, 3, 181, 182, 335, 362, 363, 384, 511, 512, 513, 3600):
        want = math.floor(2 * math.log2(n) + 1e-12)
        assert hpez.hpez_level_key_of((n, 8), None, 1, False)[2] == want, n
    cfg = hpez.make_config(3, paradigm=1, interp=0)
    assert hpez.hpez_level_key_of((64, 64, 64), cfg, 1, False)[5:7] == (0, 1)
    # same-level halves and block maps take the per-point interpolator
    cfg = hpez.make_config(3, same_level=1)
    assert hpez.hpez_level_key_of((64, 64, 64), cfg, 1, False)[5] == 3
    nb = hpez.hpez_blockmap_size((64, 64, 64), 32)
    mixed = hpez.make_config(3, blockmap=[0, 1] * (nb // 2))
    assert hpez.hpez_level_key_of((64, 64, 64), mixed, 2, False)[5] == 3
    # a uniform block map is its interpolator in compress; decompress plans
    # from the header's config
    uni = hpez.make_config(3, blockmap=[1] * nb)
    assert hpez.hpez_level_key_of((64, 64, 64), uni, 2, False)[5] == 1
    assert hpez.hpez_level_key_of((64, 64, 64), uni, 2, True)[5] == 3
    for bad in ((0, 4, 4), (8, 8, 8)):
        with pytest.raises(hpez.HpezError):
            hpez.hpez_level_key_of(bad, None, 9 if bad[0] else 1, False)


def test_table_set_get_save_load(tmp_path):
    t = hpez.Tuning()
    k1 = (3, 7, 9, 9, 1, 1, 0, 0)
    k2 = (2, 0, 11, 12, 2, 1, 0, 1)
    t.set(k1, hpez.HPEZ_FAM_LEVEL3D, (0, 8, 0), time_us=123.5)
    t.set(k2, hpez.HPEZ_FAM_FUSED, (1, 16, 64))
    t.set(k1, hpez.HPEZ_FAM_LEVEL3D, (0, 4, 0), time_us=99.25)  # replaces
    assert len(t) == 2
    v = t.get(k1)
    assert v.astuple() == (hpez.HPEZ_FAM_LEVEL3D, 0, 4, 0, 0) and v.time_us == 99.25
    assert t.get((3, 7, 9, 9, 2, 1, 0, 0)) is None
    path = str(tmp_path / "sched.txt")
    t.save(path)
    u = hpez.Tuning(path)
    assert len(u) == 2
    assert u.get(k2).astuple() == (hpez.HPEZ_FAM_FUSED, 1, 16, 64, 0)
    # load merges
    w = hpez.Tuning()
    w.set((1, 0, 0, 12, 1, 0, 0, 0), hpez.HPEZ_FAM_PASS)
    w.load(path)
    assert len(w) == 3


@pytest.mark.parametrize("line", [
    "3 7 9 9 1 1 0 0 1 0 8 0 0",             # a field missing
    "3 7 9 9 3 1 0 0 1 0 8 0 0 1.0",         # stride not a power of two
    "3 7 9 9 1 1 0 0 9 0 8 0 0 1.0",         # unknown family
    "4 7 9 9 1 1 0 0 1 0 8 0 0 1.0",         # ndim out of range
    "3 7 9 9 1 1 0 0 1 0 8 0 0 1.0 7",       # trailing field
    "3 7 9 9 1 1 0 0 1 0 -8 0 0 1.0",        # negative tile
])
def test_malformed_files_rejected(tmp_path, line):
    path = tmp_path / "bad.txt"
    path.write_text("# header\n3 7 9 9 2 1 0 0 1 0 8 0 0 1.0\n" + line + "\n")
    t = hpez.Tuning()
    with pytest.raises(hpez.HpezError):
        t.load(str(path))
    assert len(t) == 0  # nothing merged from a bad file
    with pytest.raises(hpez.HpezError):
        t.load(str(tmp_path / "missing.txt"))
    with pytest.raises(hpez.HpezError):
        t.set((3, 7, 9, 9, 1, 4, 0, 0), hpez.HPEZ_FAM_LEVEL3D)  # interp 4


def test_shipped_table_loads():
    """The searched schedules shipped with the package parse."""
    path = os.path.join(os.path.dirname(hpez.__file__), "tuning", "levels_gb300.txt")
    if not os.path.exists(path):
        pytest.skip("no shipped table")
    t = hpez.Tuning(path)
    assert len(t) > 0
