"""Host-side bookkeeping of bench.py: the algorithmic bytes per phase and
the recorded DRAM traffic, which must stand only for the kernel sources it
was measured on."""
import json
import math
import os

import bench


def test_phase_bytes():
    shape, A = (64, 64, 64), 32
    N = math.prod(shape)
    gs = bench.grid_sizes(shape, A)
    assert gs[0] == N and gs[1] == 32 ** 3 and gs[-1] == 2 ** 3  # anchors 0, 32 per side
    n_s, n_c = gs[0], gs[1]
    # finest level, compress: new x, coarse recon, coarse codes, codes out
    assert bench.phase_bytes("level1", shape, A, 0) == 4 * (n_s - n_c) + 4 * n_c + 2 * n_s + 2 * n_c
    assert bench.phase_bytes("dlevel1", shape, A, 0) == 2 * (n_s - n_c) + 4 * n_c + 4 * n_s
    assert bench.phase_bytes("pack", shape, A, 1000) == 2 * N + 1000
    assert bench.phase_bytes("range", shape, A, 0) == 4 * N
    # the Lorenzo pass reads 4 N (or 2 N) and writes 2 N (or 4 N)
    assert bench.phase_bytes("level1", shape, A, 0, lorenzo=True) == 6 * N
    assert bench.phase_bytes("dlevel1", shape, A, 0, lorenzo=True) == 6 * N


def test_recorded_traffic_keyed_to_sources(tmp_path, monkeypatch):
    """Every recorded figure carries the hash of its kernel's sources; a
    changed source makes it unavailable (None), never a stale number."""
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for phase, e in d["phases"].items():
        assert phase in bench.PHASE_SOURCES, phase
        assert e["bytes"] > 0 and len(e["src_hash"]) == 16
        got = bench.ncu_traffic(phase)
        assert got in (None, e["bytes"])
    # a figure recorded on other sources is not reported
    fake_root = tmp_path
    (fake_root / "profiles").mkdir()
    (fake_root / "paper_2311_12133_gb300").symlink_to(
        os.path.join(bench.ROOT, "paper_2311_12133_gb300"))
    d2 = {"phases": {"level1": {"bytes": 123, "src_hash": "0" * 16}}}
    (fake_root / "profiles" / "traffic.json").write_text(json.dumps(d2))
    monkeypatch.setattr(bench, "ROOT", str(fake_root))
    assert bench.ncu_traffic("level1") is None
    d2["phases"]["level1"]["src_hash"] = bench.src_hash(bench.PHASE_SOURCES["level1"])
    (fake_root / "profiles" / "traffic.json").write_text(json.dumps(d2))
    assert bench.ncu_traffic("level1") == 123
    assert bench.ncu_traffic("no_such_phase") is None
