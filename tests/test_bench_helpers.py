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


def test_step_stats_and_percentile():
    ms = [float(v) for v in range(1, 101)]
    st = bench.step_stats(ms)
    assert st["median"] == 50.5 and st["p99"] == 99.0 and st["max"] == 100.0
    assert bench.percentile([3.0, 1.0, 2.0], 50) == 2.0
    assert bench.step_stats([2.0])["p99"] == 2.0


def test_clock_samples_by_window(tmp_path):
    """Samples are picked out by their timestamps: the timed window and the
    loaded stretch, with throttle reasons only from the loaded stretch."""
    rows = [
        "2026/12/04 10:00:00.000, GPU-abc, 900, 2070, 100, 0x0, Not Active, Not Active, Not Active, Active",
        "2026/12/04 10:00:01.000, GPU-abc, 2000, 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2026/12/04 10:00:02.000, GPU-abc, 2070, 2070, 950, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2026/12/04 10:00:02.010, GPU-xyz, 100, 2070, 950, 0x0, Active, Not Active, Not Active, Not Active",
    ]
    p = tmp_path / "clk.csv"
    p.write_text("\n".join(rows) + "\n")
    t = bench.ClockSampler.parse_time

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            pass
    s = bench.ClockSampler("GPU-abc")
    s.proc, s.path = Done(), str(p)
    c = s.stop(timed=(t("2026/12/04 10:00:01.900"), t("2026/12/04 10:00:02.000")),
               loaded=(t("2026/12/04 10:00:00.500"), t("2026/12/04 10:00:02.000")))
    assert c["samples"] == 2 and c["samples_timed"] == 1
    assert c["sm_mhz"] == 2035.0 and c["sm_mhz_timed"] == 2070.0
    assert c["reasons"] == []  # the power-cap sample lies before the loaded stretch


def test_psnr_of_uniform_error():
    import numpy as np
    import torch
    x = torch.linspace(0, 1, 1 << 16, dtype=torch.float32)
    e = torch.from_numpy(np.random.default_rng(0).uniform(-1e-3, 1e-3, x.numel())
                         .astype(np.float32))
    y = x + e
    # uniform error on [-e, e]: MSE ~ e^2 / 3, range 1
    want = -10 * math.log10((1e-3) ** 2 / 3)
    assert abs(bench.psnr_db(x, y) - want) < 0.1
    assert bench.psnr_db(x, x.clone()) == float("inf")
