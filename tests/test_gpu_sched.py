"""Level schedules of the batched form: the offline search, and batches run
under searched and forced schedule tables.  A schedule changes how the GPU
runs a level, never what it computes, so every stream and field must equal
the oracle's under any table."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_12133_gb300 import build as B
    B.build()
    from paper_2311_12133_gb300 import hpez
    ctx = hpez.Context(0)
    yield ctx
    hpez.hpez_use_tuning(ctx.handle, None)
    ctx.close()


def _mix():
    from paper_2311_12133_gb300 import fields
    return [
        (fields.make("grf", (40, 48, 64), 1), 1e-3, None),
        (fields.make("bumps", (36, 40, 44), 2), 1e-3, dict(paradigm=1, interp=0)),
        (fields.make("lognormal", (30, 34, 50), 3), 1e-2, dict(paradigm=1, interp=1)),
        (fields.make("climate2d", (90, 130), 4), 1e-3, None),
        (fields.make("grf", (33, 20, 47), 5), 1e-4, dict(interp=2)),
    ]


@pytest.fixture(scope="module")
def expected(oracle):
    from oracle import oracle as O
    out = []
    for x, eb, kw in _mix():
        ocfg = O.make_config(x.ndim, **kw) if kw else None
        s, _, _, recon = oracle.compress(x, eb, 1, ocfg, want_recon=True)
        out.append((s, recon))
    return out


def _levels(hpez, shape, cfg):
    """The level count of a field (key_of refuses a level beyond it)."""
    L = 0
    while True:
        try:
            hpez.hpez_level_key_of(shape, cfg, L + 1, False)
        except hpez.HpezError:
            return L
        L += 1


def _table_for(hpez, fam, tile=(0, 0, 0), chunks=0):
    """A table mapping every level of every field of the mix (both
    directions) to one schedule."""
    t = hpez.Tuning()
    for x, eb, kw in _mix():
        cfg = hpez.make_config(x.ndim, **kw) if kw else None
        for l in range(1, _levels(hpez, x.shape, cfg) + 1):
            for d in (False, True):
                t.set(hpez.hpez_level_key_of(x.shape, cfg, l, d), fam, tile, chunks)
    return t


def _run_and_check(gpu, expected):
    import torch
    from paper_2311_12133_gb300 import hpez
    mix = _mix()
    xs = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x, _, _ in mix]
    cfgs = [hpez.make_config(x.ndim, **kw) if kw else None for x, _, kw in mix]
    b = hpez.Batch(gpu, fields=[(xs[i], mix[i][1], 1, cfgs[i]) for i in range(len(mix))])
    b.run(graph=True)
    sizes, st = b.results()
    assert st == [0] * len(mix)
    for i in range(len(mix)):
        assert b.outs[i][:sizes[i]].cpu().numpy().tobytes() == expected[i][0], i
    b.close()
    bufs = [torch.from_numpy(np.frombuffer(s, np.uint8).copy()).cuda() for s, _ in expected]
    d = hpez.Batch(gpu, streams=[(bufs[i], len(expected[i][0]), expected[i][0][:512])
                                 for i in range(len(mix))])
    d.run()
    _, st = d.results()
    assert st == [0] * len(mix)
    for i in range(len(mix)):
        assert d.outs[i].cpu().numpy().tobytes() == expected[i][1].tobytes(), i
    d.close()


@pytest.mark.parametrize("sched", [
    ("LEVEL3D", (0, 2, 0), 0), ("LEVEL3D", (0, 32, 0), 0),
    ("MD3W", (0, 0, 0), 1), ("MD3W", (0, 0, 0), 3),
    ("MD3", (0, 2, 0), 0), ("MD3", (0, 32, 0), 0),
    ("FUSED", (4, 8, 64), 0), ("FUSED", (1, 2, 512), 0), ("FUSED", (1, 32, 64), 0),
    ("PASS", (0, 0, 0), 0)])
def test_forced_schedules_equal_oracle(gpu, expected, sched):
    """Every level of every field forced to one schedule (levels that cannot
    run it keep the fixed rules)."""
    from paper_2311_12133_gb300 import hpez
    fam, tile, chunks = sched
    t = _table_for(hpez, getattr(hpez, "HPEZ_FAM_" + fam), tile, chunks)
    hpez.hpez_use_tuning(gpu.handle, t)
    try:
        _run_and_check(gpu, expected)
    finally:
        hpez.hpez_use_tuning(gpu.handle, None)


def test_search_then_tuned_batch(gpu, expected, tmp_path):
    """The search fills an entry for every level and direction of each
    searched class; a batch under the saved and reloaded table equals the
    oracle."""
    import torch
    from paper_2311_12133_gb300 import hpez
    t = hpez.Tuning()
    for x, eb, kw in _mix():
        cfg = hpez.make_config(x.ndim, **kw) if kw else None
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        t.search(gpu, xd, eb, 1, cfg, copies=2, reps=1)
        for l in range(1, _levels(hpez, x.shape, cfg) + 1):
            for d in (False, True):
                v = t.get(hpez.hpez_level_key_of(x.shape, cfg, l, d))
                assert v is not None and v.time_us > 0
                assert 1 <= v.family <= 5
    path = str(tmp_path / "levels.txt")
    t.save(path)
    hpez.hpez_use_tuning(gpu.handle, hpez.Tuning(path))
    try:
        _run_and_check(gpu, expected)
    finally:
        hpez.hpez_use_tuning(gpu.handle, None)


def test_shipped_table_batch_equals_oracle(gpu, oracle):
    """The searched table shipped with the package, on the smallest fields
    of the 64-field benchmark mix (both configurations it was searched
    for): streams and fields equal the oracle's."""
    import os
    import torch
    from oracle import oracle as O
    from paper_2311_12133_gb300 import autotune, fields, hpez
    if not os.path.exists(autotune.SHIPPED):
        pytest.skip("no shipped table")
    t = hpez.Tuning(autotune.SHIPPED)
    specs = sorted(autotune.mix_specs(), key=lambda s: int(np.prod(s[1])))[:8]
    hpez.hpez_use_tuning(gpu.handle, t)
    try:
        xs, args, want = [], [], []
        for kind, shape, seed, eb, kw in specs:
            x = fields.make(kind, shape, seed)
            xd = torch.from_numpy(x).cuda()
            xs.append(xd)
            args.append((xd, eb, 1, hpez.make_config(x.ndim, **kw) if kw else None))
            st, _, _, recon = oracle.compress(x, eb, 1, O.make_config(x.ndim, **kw) if kw
                                              else None, want_recon=True)
            want.append((st, recon))
            assert t.get(hpez.hpez_level_key_of(shape, args[-1][3], 1, False)) is not None
        b = hpez.Batch(gpu, fields=args)
        b.run(graph=True)
        sizes, status = b.results()
        assert status == [0] * len(specs)
        for i in range(len(specs)):
            assert b.outs[i][:sizes[i]].cpu().numpy().tobytes() == want[i][0], i
        b.close()
        bufs = [torch.from_numpy(np.frombuffer(w, np.uint8).copy()).cuda() for w, _ in want]
        d = hpez.Batch(gpu, streams=[(bufs[i], len(want[i][0]), want[i][0][:512])
                                     for i in range(len(specs))])
        d.run(graph=True)
        _, st = d.results()
        assert st == [0] * len(specs)
        for i in range(len(specs)):
            assert d.outs[i].cpu().numpy().tobytes() == want[i][1].tobytes(), i
        d.close()
    finally:
        hpez.hpez_use_tuning(gpu.handle, None)


@pytest.mark.parametrize("chunks", [1, 3, 7])
def test_single_calls_follow_the_table(gpu, oracle, chunks):
    """The single-field calls take a level's tile shape and chunk count from
    the table: the warp-strip level with several chunk counts, the 3D and
    fused level kernels with other tiles; streams and fields equal the
    oracle's."""
    import torch
    from oracle import oracle as O
    from paper_2311_12133_gb300 import fields, hpez
    cases = [(fields.make("grf", (40, 48, 64), 31), dict(paradigm=1, interp=0)),
             (fields.make("bumps", (36, 40, 44), 32), None),
             (fields.make("climate2d", (90, 130), 33), None)]
    t = hpez.Tuning()
    for x, kw in cases:
        cfg = hpez.make_config(x.ndim, **kw) if kw else None
        for l in range(1, _levels(hpez, x.shape, cfg) + 1):
            for d in (False, True):
                k = hpez.hpez_level_key_of(x.shape, cfg, l, d)
                if kw:
                    t.set(k, hpez.HPEZ_FAM_MD3W if l == 1 else hpez.HPEZ_FAM_MD3,
                          (0, 4, 0), chunks)
                elif x.ndim == 3:
                    t.set(k, hpez.HPEZ_FAM_LEVEL3D, (0, 2 * chunks, 0))
                else:
                    t.set(k, hpez.HPEZ_FAM_FUSED, (1, 2 * chunks, 64))
    hpez.hpez_use_tuning(gpu.handle, t)
    try:
        for x, kw in cases:
            cfg = hpez.make_config(x.ndim, **kw) if kw else None
            want, _, _, _ = oracle.compress(x, 1e-3, 1, O.make_config(x.ndim, **kw) if kw
                                            else None)
            buf, size = gpu.compress(torch.from_numpy(x).cuda(), 1e-3, 1, cfg)
            assert buf[:size].cpu().numpy().tobytes() == want
            y = gpu.decompress(buf, size).cpu().numpy()
            assert y.tobytes() == oracle.decompress(want).tobytes()
    finally:
        hpez.hpez_use_tuning(gpu.handle, None)
