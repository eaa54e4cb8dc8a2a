"""The C-ABI library builds, loads and exports every entry point that
include/hpez.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "hpez.h")).read()
    return sorted(set(re.findall(r"HPEZ_API\s+[\w\s\*]+?\b(hpez_\w+)\s*\(", txt)))


def test_header_declares_entry_points():
    syms = declared_symbols()
    for s in ("hpez_create", "hpez_compress", "hpez_decompress", "hpez_inspect"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_2311_12133_gb300 import build as B
    from paper_2311_12133_gb300 import hpez
    path = B.build()
    lib = ctypes.CDLL(path)
    for s in declared_symbols():
        assert hasattr(lib, s), s
    assert set(hpez.exported_symbols()) <= set(declared_symbols())


def test_host_side_calls_without_gpu():
    """Pure host entry points work without a device."""
    from paper_2311_12133_gb300 import hpez
    cfg = hpez.hpez_default_config(3)
    assert cfg.anchor_stride == 32 and cfg.chunk_syms == 16384
    assert hpez.hpez_compress_bound((128, 128, 128)) > 4 * 128 ** 3
    assert hpez.hpez_strerror(-4).startswith("corrupt")
    import pytest
    with pytest.raises(hpez.HpezError):
        hpez.hpez_inspect(b"\0" * 512)
