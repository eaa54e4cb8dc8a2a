"""The batched and served forms against the single-field path and the
oracle.

Both forms run the single-field operations, only grouped into shared
launches, so every stream must equal the one hpez_compress writes (and the
oracle's), and every decompressed field the single-field result, byte for
byte -- alone or in any mix.
"""
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
    ctx.close()


def _mix(seed=0):
    """Fields of mixed dimension, shape, bound mode and configuration,
    including the per-pass path (multi-dimensional paradigm), a block map,
    a frozen dimension, 1D and a constant field."""
    from paper_2311_12133_gb300 import fields, hpez
    rng = np.random.default_rng(seed)
    out = []
    out.append((fields.make("bumps", (40, 36, 33), 1), 1e-3, 1, None))
    out.append((fields.make("grf", (64, 64, 64), 2), 1e-2, 1, None))
    out.append((fields.make("climate2d", (90, 130), 3), 1e-3, 1, None))
    out.append((fields.make("grf", (17, 300), 4), 1e-4, 1, None))
    out.append((fields.make("lognormal", (30, 41, 52), 5), 0.05, 0, None))
    out.append((np.cumsum(rng.normal(0, 1, 3000)).astype(np.float32), 1e-3, 1, None))
    out.append((fields.make("grf", (33, 40, 47), 6), 1e-3, 1,
                dict(paradigm=1, interp=2)))
    nb = hpez.hpez_blockmap_size((48, 50, 37), 16)
    out.append((fields.make("bumps", (48, 50, 37), 7), 1e-3, 1,
                dict(block_size=16, blockmap=rng.choice([0, 1, 2, 5, 6], nb))))
    out.append((fields.make("grf", (36, 40, 44), 8), 1e-3, 1,
                dict(frozen_dim=1, same_level=1)))
    out.append((np.full((20, 30), 2.5, np.float32), 1e-3, 1, None))
    out.append((fields.make("aniso", (10, 96, 96), 9), 1e-3, 1,
                dict(interp=0, anchor_stride=16)))
    return out


def _cfgs(x, kw):
    from oracle import oracle as O
    from paper_2311_12133_gb300 import hpez
    if kw is None:
        return None, None
    return hpez.make_config(x.ndim, **kw), O.make_config(x.ndim, **kw)


def test_batch_compress_equals_single_and_oracle(gpu, oracle):
    import torch
    from paper_2311_12133_gb300 import hpez
    mix = _mix()
    xs, fields_arg, ocfgs = [], [], []
    for x, eb, mode, kw in mix:
        g, o = _cfgs(x, kw)
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        xs.append(xd)
        fields_arg.append((xd, eb, mode, g))
        ocfgs.append(o)
    b = hpez.Batch(gpu, fields=fields_arg)
    b.run()
    sizes, status = b.results()
    assert status == [0] * len(mix)
    launches, ticks = b.launch_count()
    assert launches < 4 * ticks
    streams = []
    for i, (x, eb, mode, kw) in enumerate(mix):
        got = b.outs[i][:sizes[i]].cpu().numpy().tobytes()
        buf, size = gpu.compress(xs[i], eb, mode, fields_arg[i][3])
        assert got == buf[:size].cpu().numpy().tobytes(), i
        want, _, _, _ = oracle.compress(x, eb, mode, ocfgs[i])
        assert got == want, i
        streams.append(got)
    # a second run and a graph replay give the same bytes
    b.run(graph=True)
    b.run(graph=True)
    sizes2, status2 = b.results()
    assert sizes2 == sizes and status2 == status
    for i in range(len(mix)):
        assert b.outs[i][:sizes[i]].cpu().numpy().tobytes() == streams[i]
    b.close()

    # batched decompress of the same streams
    bufs = [torch.from_numpy(np.frombuffer(s_, np.uint8).copy()).cuda() for s_ in streams]
    d = hpez.Batch(gpu, streams=[(bufs[i], len(streams[i]), streams[i][:512])
                                 for i in range(len(streams))])
    d.run(graph=True)
    _, st = d.results()
    assert st == [0] * len(streams)
    for i in range(len(streams)):
        y = gpu.decompress(bufs[i], len(streams[i])).cpu().numpy()
        assert d.outs[i].cpu().numpy().tobytes() == y.tobytes(), i
        assert y.tobytes() == oracle.decompress(streams[i]).tobytes(), i
    d.close()


def _md_mix():
    """Fields whose levels run the multi-dimensional kernels of the batched
    form: warp strips at the finest level (rows of an even length), the
    even/odd-plane launches elsewhere, every interpolator."""
    from paper_2311_12133_gb300 import fields
    return [
        (fields.make("grf", (40, 48, 64), 11), 1e-3, 1, dict(paradigm=1, interp=0)),
        (fields.make("bumps", (30, 34, 50), 12), 1e-3, 1, dict(paradigm=1, interp=1)),
        (fields.make("lognormal", (26, 31, 44), 13), 1e-2, 1, dict(paradigm=1, interp=2)),
        (fields.make("grf", (65, 20, 36), 14), 1e-4, 1, dict(paradigm=1, interp=0)),
        (fields.make("grf", (33, 40, 47), 6), 1e-3, 1, dict(paradigm=1, interp=2)),
        (fields.make("bumps", (40, 36, 33), 1), 1e-3, 1, None),
        (fields.make("climate2d", (90, 130), 3), 1e-3, 1, None),
    ]


@pytest.mark.parametrize("warp_levels,batch_ctas", [(1, 0), (0, 5), (1, 3)])
def test_batch_md_levels_and_persistent_walk(gpu, oracle, warp_levels, batch_ctas):
    """Multi-dimensional levels in the batch, and persistent level launches
    capped at a few CTAs so each walks many tiles of several fields: the
    streams and fields equal the oracle's."""
    import torch
    from paper_2311_12133_gb300 import hpez
    hpez.hpez_set_option(gpu.handle, hpez.HPEZ_OPT_WARP_LEVELS, warp_levels)
    hpez.hpez_set_option(gpu.handle, hpez.HPEZ_OPT_BATCH_CTAS, batch_ctas)
    try:
        mix = _md_mix()
        xs, fields_arg, ocfgs = [], [], []
        for x, eb, mode, kw in mix:
            g, o = _cfgs(x, kw)
            xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
            xs.append(xd)
            fields_arg.append((xd, eb, mode, g))
            ocfgs.append(o)
        b = hpez.Batch(gpu, fields=fields_arg)
        b.run(graph=True)
        sizes, status = b.results()
        assert status == [0] * len(mix)
        streams = []
        for i, (x, eb, mode, kw) in enumerate(mix):
            got = b.outs[i][:sizes[i]].cpu().numpy().tobytes()
            want, _, _, recon = oracle.compress(x, eb, mode, ocfgs[i], want_recon=True)
            assert got == want, i
            streams.append((got, recon))
        b.close()
        bufs = [torch.from_numpy(np.frombuffer(s_, np.uint8).copy()).cuda()
                for s_, _ in streams]
        d = hpez.Batch(gpu, streams=[(bufs[i], len(streams[i][0]), streams[i][0][:512])
                                     for i in range(len(streams))])
        d.run(graph=True)
        _, st = d.results()
        assert st == [0] * len(streams)
        for i in range(len(streams)):
            assert d.outs[i].cpu().numpy().tobytes() == streams[i][1].tobytes(), i
        d.close()
    finally:
        hpez.hpez_set_option(gpu.handle, hpez.HPEZ_OPT_WARP_LEVELS, 1)
        hpez.hpez_set_option(gpu.handle, hpez.HPEZ_OPT_BATCH_CTAS, 0)


@pytest.mark.parametrize("lorenzo_ctas", [0, 4])
def test_batch_lorenzo_fields_equal_oracle(gpu, oracle, lorenzo_ctas):
    """Lorenzo-predictor fields (Sec. 6.5) of order 1 and 2, 1D to 3D, in a
    batch with interpolation fields: streams and fields equal the oracle's
    (with few CTAs, each streams many blocks)."""
    import torch
    from paper_2311_12133_gb300 import fields, hpez
    mix = [
        (fields.make("grf", (64, 64, 64), 21), 1e-3, dict(predictor=1)),
        (fields.make("bumps", (40, 50, 36), 22), 1e-3, dict(predictor=2)),
        (fields.make("climate2d", (130, 200), 23), 1e-3, dict(predictor=1)),
        (fields.make("grf", (70, 90, 100), 24), 1e-4, dict(predictor=2)),
        (np.cumsum(np.random.default_rng(5).normal(0, 1, 5000)).astype(np.float32), 1e-3,
         dict(predictor=1)),
        (fields.make("grf", (40, 48, 64), 25), 1e-3, None),
    ]
    hpez.hpez_set_option(gpu.handle, hpez.HPEZ_OPT_LORENZO_CTAS, lorenzo_ctas)
    try:
        xs, args, want = [], [], []
        for x, eb, kw in mix:
            xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
            xs.append(xd)
            args.append((xd, eb, 1, hpez.make_config(x.ndim, **kw) if kw else None))
            ocfg = oracle.make_config(x.ndim, **kw) if kw else None
            st, _, _, recon = oracle.compress(x, eb, 1, ocfg, want_recon=True)
            want.append((st, recon))
        b = hpez.Batch(gpu, fields=args)
        b.run(graph=True)
        sizes, status = b.results()
        assert status == [0] * len(mix)
        for i in range(len(mix)):
            assert b.outs[i][:sizes[i]].cpu().numpy().tobytes() == want[i][0], i
        b.close()
        bufs = [torch.from_numpy(np.frombuffer(w, np.uint8).copy()).cuda() for w, _ in want]
        d = hpez.Batch(gpu, streams=[(bufs[i], len(want[i][0]), want[i][0][:512])
                                     for i in range(len(mix))])
        d.run()
        _, st = d.results()
        assert st == [0] * len(mix)
        for i in range(len(mix)):
            assert d.outs[i].cpu().numpy().tobytes() == want[i][1].tobytes(), i
        d.close()
    finally:
        hpez.hpez_set_option(gpu.handle, hpez.HPEZ_OPT_LORENZO_CTAS, 0)


def test_batch_levels_share_launches(gpu):
    """Fields with different numbers of levels run each level in the same
    launches: the ticks are the distinct op keys, fewer than the ops of the
    longest request plus the extra levels of the others."""
    import torch
    from paper_2311_12133_gb300 import fields, hpez
    shapes = [(40, 48, 64), (100, 90, 80), (20, 24, 28), (130, 150)]
    xs = [torch.from_numpy(fields.make("grf", sh, i)).cuda() for i, sh in enumerate(shapes)]
    b = hpez.Batch(gpu, fields=[(x, 1e-3, 1, None) for x in xs])
    b.run()
    sizes, st = b.results()
    assert st == [0] * len(xs)
    launches, ticks = b.launch_count()
    # 4 ops before the sweep, one op per level (5 levels at the 3D anchor
    # stride 32, 6 at the 2D stride 64: the level ticks are the 2D field's),
    # 11 ops after the sweep
    assert ticks == 4 + 6 + 11
    for i, x in enumerate(xs):
        buf, size = gpu.compress(x, 1e-3)
        assert b.outs[i][:sizes[i]].cpu().numpy().tobytes() == buf[:size].cpu().numpy().tobytes()
    b.close()


def test_batch_errors(gpu):
    import torch
    from paper_2311_12133_gb300 import hpez
    x = torch.rand((20, 20), device="cuda")
    with pytest.raises(hpez.HpezError) as e:
        hpez.Batch(gpu, fields=[(x, 1e-3, 1, None), (x, -1.0, 1, None)])
    assert e.value.code == -1
    # a corrupt stream is reported per request, the others succeed
    xs = [torch.rand((30, 40), device="cuda") for _ in range(3)]
    b = hpez.Batch(gpu, fields=[(v, 1e-3, 1, None) for v in xs])
    b.run()
    sizes, st = b.results()
    assert st == [0, 0, 0]
    bufs = [b.outs[i][:sizes[i]].clone() for i in range(3)]
    hdrs = [bufs[i][:512].cpu().numpy().tobytes() for i in range(3)]
    raw = bufs[1].cpu().numpy()
    # swap the first two code-table symbols: the table is no longer
    # ascending, which the decoder rejects
    ot = int(np.frombuffer(raw[272:280].tobytes(), np.uint64)[0])
    raw[[ot, ot + 1, ot + 2, ot + 3]] = raw[[ot + 2, ot + 3, ot, ot + 1]]
    bufs[1] = torch.from_numpy(raw).cuda()
    d = hpez.Batch(gpu, streams=[(bufs[i], sizes[i], hdrs[i]) for i in range(3)])
    d.run()
    _, st = d.results()
    assert st[0] == 0 and st[2] == 0 and st[1] == -4
    b.close()
    d.close()


def test_context_closes_its_batches_first(gpu):
    """Closing a context destroys the batches and servers made on it first,
    and leaves no CUDA error behind for the next call on another context."""
    import torch
    from paper_2311_12133_gb300 import hpez
    c2 = hpez.Context(0)
    x = torch.rand((30, 40, 50), device="cuda")
    b = hpez.Batch(c2, fields=[(x, 1e-3, 1, None)])
    b.run()
    srv = hpez.Server(c2, 1 << 26, 2)
    c2.close()
    assert b.handle == 0 and srv.handle == 0
    del b, srv
    import gc
    gc.collect()
    buf, size = gpu.compress(x, 1e-3)
    y = gpu.decompress(buf, size)
    assert (y - x).abs().max().item() <= 1e-3 * (x.max() - x.min()).item()


def _served_mix(gpu, oracle, mix, budget, slots, seed):
    """Serve every field of `mix` twice (once compressed, once its stream
    decompressed), submitting a few requests between steps so that later
    requests join running ones: every result equals the oracle's stream or
    reconstruction and the single call's."""
    import torch
    from paper_2311_12133_gb300 import hpez
    single = []
    for x, eb, mode, kw in mix:
        g, o = _cfgs(x, kw)
        want, _, _, recon = oracle.compress(x, eb, mode, o, want_recon=True)
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        buf, size = gpu.compress(xd, eb, mode, g)
        s_ = buf[:size].cpu().numpy().tobytes()
        y = gpu.decompress(buf, size).cpu().numpy()
        assert s_ == want
        want_y = oracle.decompress(want)
        assert y.tobytes() == want_y.tobytes()
        single.append((s_, want_y))
    srv = hpez.Server(gpu, budget, max_slots=slots)
    pending = {}
    order = list(range(len(mix))) * 2
    rng = np.random.default_rng(seed)
    rng.shuffle(order)
    k = 0
    served = 0
    max_active = 0
    while k < len(order) or pending:
        for _ in range(int(rng.integers(0, 4))):
            if k >= len(order):
                break
            i = order[k]
            x, eb, mode, kw = mix[i]
            if k % 2 == 0:
                g, _ = _cfgs(x, kw)
                rid, out = srv.submit_compress(np.ascontiguousarray(x), eb, mode, g)
                pending[rid] = ("c", i, out)
            else:
                s_ = single[i][0]
                h = np.frombuffer(s_, np.uint8).copy()
                rid, out = srv.submit_decompress(h, len(s_))
                pending[rid] = ("d", i, out)
            k += 1
        srv.step()
        max_active = max(max_active, srv.stats()["active"])
        for rid, st, size, lat in srv.poll():
            kind, i, out = pending.pop(rid)
            assert st == 0, (kind, i, st)
            if kind == "c":
                assert out[:size].tobytes() == single[i][0], i
            else:
                assert out.tobytes() == single[i][1].tobytes(), i
            assert lat >= 0
            served += 1
    stats = srv.stats()
    assert stats["active"] == 0 and stats["queued"] == 0 and stats["used_bytes"] == 0
    srv.close()
    assert served == len(order)
    return max_active


def test_server_results_equal_oracle_under_load(gpu, oracle):
    """Thirty fields of 0.5-8 MB from the workload generators, rel eb from
    {1e-2, 1e-3, 1e-4}, served through eight slots under a budget that
    queues requests: several requests are in flight at once and every
    served stream and field equals the oracle's."""
    from paper_2311_12133_gb300 import fields
    rng = np.random.default_rng(11)
    mix = []
    kinds = ["bumps", "grf", "lognormal", "aniso", "climate2d"]
    for j in range(30):
        kind = kinds[j % 5]
        npts = int(np.exp(rng.uniform(np.log(1.3e5), np.log(2.1e6))))
        if kind == "climate2d":
            ny = max(16, int(np.sqrt(npts / 2)))
            shape = (ny, max(16, npts // ny))
        else:
            side = max(12, int(round(npts ** (1 / 3))))
            shape = (side, side + int(rng.integers(-4, 5)), side + int(rng.integers(0, 9)))
        eb = [1e-2, 1e-3, 1e-4][int(rng.integers(0, 3))]
        mix.append((fields.make(kind, shape, 40 + j), eb, 1, None))
    max_active = _served_mix(gpu, oracle, mix, 96 << 20, 8, 3)
    assert max_active >= 2


def test_server_results_equal_single_calls(gpu, oracle):
    """Requests of mixed size and kind, submitted while others run, under a
    budget that forces queueing: every result equals the single call's and
    the oracle's."""
    _served_mix(gpu, oracle, _mix(1), 48 << 20, 4, 0)


def test_server_rejects_oversized(gpu):
    from paper_2311_12133_gb300 import hpez
    srv = hpez.Server(gpu, 1 << 20, max_slots=2)
    x = np.zeros((128, 128, 64), np.float32)
    with pytest.raises(hpez.HpezError) as e:
        srv.submit_compress(x, 1e-3)
    assert e.value.code == -10
    srv.close()
