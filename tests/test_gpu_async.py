"""hpez_compress_async / hpez_decompress_async: the single-field launch
sequences with no host synchronization, the outcome written on the device.
Their streams and fields must equal the synchronous calls' (and the
oracle's) byte for byte, errors must arrive as the device status, and a
call that needs no scratch growth must replay from a CUDA graph."""
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


def _cases():
    from paper_2311_12133_gb300 import fields
    rng = np.random.default_rng(7)
    return [
        (fields.make("grf", (48, 52, 64), 1), 1e-3, None),
        (fields.make("bumps", (40, 44, 36), 2), 1e-3, dict(paradigm=1, interp=0)),
        (fields.make("climate2d", (120, 170), 3), 1e-3, dict(same_level=1)),
        (fields.make("grf", (64, 64, 64), 4), 1e-3, dict(predictor=1)),
        (fields.make("grf", (30, 40, 50), 5), 1e-3, dict(interp=3)),
        (np.cumsum(rng.normal(0, 1, 4000)).astype(np.float32), 1e-2, None),
        (np.full((30, 40), 1.5, np.float32), 1e-3, None),                 # constant field
        (np.zeros((16, 16, 64), np.float32) + np.float32(0.25) *
         (np.arange(64, dtype=np.float32) % 2), 10.0, None),               # one-symbol table
    ]


def test_async_equals_sync_and_oracle(gpu, oracle):
    import torch
    from paper_2311_12133_gb300 import hpez
    s = torch.cuda.current_stream().cuda_stream
    for i, (x, eb, kw) in enumerate(_cases()):
        cfg = hpez.make_config(x.ndim, **kw) if kw else None
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        cap = hpez.hpez_compress_bound(x.shape)
        out = torch.empty(cap, dtype=torch.uint8, device="cuda")
        sz = torch.full((1,), 7, dtype=torch.int64, device="cuda")
        st0 = torch.full((1,), -99, dtype=torch.int32, device="cuda")
        hpez.hpez_compress_async(gpu.handle, xd.data_ptr(), x.shape, 1, eb, cfg, out.data_ptr(),
                                 cap, sz.data_ptr(), st0.data_ptr(), s)
        size, status = sz.item(), st0.item()
        assert status == 0, i
        buf, ref = gpu.compress(xd, eb, 1, cfg)
        assert size == ref
        got = out[:size].cpu().numpy().tobytes()
        assert got == buf[:ref].cpu().numpy().tobytes(), i
        ocfg = oracle.make_config(x.ndim, **kw) if kw else None
        want, _, _, _ = oracle.compress(x, eb, 1, ocfg)
        assert got == want, i
        recon = oracle.decompress(want)
        y = torch.full(x.shape, float("nan"), dtype=torch.float32, device="cuda")
        st = torch.full((1,), -99, dtype=torch.int32, device="cuda")
        hpez.hpez_decompress_async(gpu.handle, out.data_ptr(), size, got[:512], y.data_ptr(),
                                   y.numel(), st.data_ptr(), s)
        assert st.item() == 0, i
        assert y.cpu().numpy().tobytes() == recon.tobytes(), i


def test_async_errors_on_the_device(gpu):
    import torch
    from paper_2311_12133_gb300 import hpez
    s = torch.cuda.current_stream().cuda_stream
    x = torch.rand((40, 40, 40), device="cuda")
    # a NaN under a relative bound: found by the range kernel
    xb = x.clone()
    xb[3, 4, 5] = float("nan")
    cap = hpez.hpez_compress_bound(x.shape)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    sz = torch.full((1,), 7, dtype=torch.int64, device="cuda")
    st0 = torch.zeros(1, dtype=torch.int32, device="cuda")
    hpez.hpez_compress_async(gpu.handle, xb.data_ptr(), x.shape, 1, 1e-3, None, out.data_ptr(),
                             cap, sz.data_ptr(), st0.data_ptr(), s)
    assert sz.item() == 0 and st0.item() == -2
    # a corrupt stream: its code table out of order
    buf, size = gpu.compress(x, 1e-3)
    raw = buf[:size].cpu().numpy().copy()
    ot = int(np.frombuffer(raw[272:280].tobytes(), np.uint64)[0])
    raw[[ot, ot + 1, ot + 2, ot + 3]] = raw[[ot + 2, ot + 3, ot, ot + 1]]
    bad = torch.from_numpy(raw).cuda()
    y = torch.empty_like(x)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    hpez.hpez_decompress_async(gpu.handle, bad.data_ptr(), size, raw[:512].tobytes(),
                               y.data_ptr(), y.numel(), st.data_ptr(), s)
    assert st.item() == -4
    # the context stays usable
    ref = gpu.decompress(buf, size)
    hpez.hpez_decompress_async(gpu.handle, buf.data_ptr(), size,
                               buf[:512].cpu().numpy().tobytes(), y.data_ptr(), y.numel(),
                               st.data_ptr(), s)
    assert st.item() == 0 and torch.equal(y, ref)
    # refused on the host: a block map in the config
    nb = hpez.hpez_blockmap_size((40, 40, 40), 32)
    with pytest.raises(hpez.HpezError) as e:
        hpez.hpez_compress_async(gpu.handle, x.data_ptr(), x.shape, 1, 1e-3,
                                 hpez.make_config(3, blockmap=[1] * nb), out.data_ptr(), cap,
                                 sz.data_ptr(), st0.data_ptr(), s)
    assert e.value.code == -8


def test_async_calls_replay_from_a_graph(gpu):
    """After a warm-up call has sized the scratch, the compress of a field
    and the decompress of a stream are captured once and replayed: new
    input values in the same buffer give the synchronous call's stream."""
    import torch
    from paper_2311_12133_gb300 import fields, hpez
    shape = (64, 72, 80)
    x = torch.from_numpy(fields.make("grf", shape, 11)).cuda()
    cap = hpez.hpez_compress_bound(shape)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    sz = torch.zeros(1, dtype=torch.int64, device="cuda")
    st0 = torch.zeros(1, dtype=torch.int32, device="cuda")
    cs = torch.cuda.Stream()
    with torch.cuda.stream(cs):
        # warm-up: scratch and kernel attributes
        hpez.hpez_compress_async(gpu.handle, x.data_ptr(), shape, 0, 1e-3, None, out.data_ptr(),
                                 cap, sz.data_ptr(), st0.data_ptr(), cs.cuda_stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cs):
        hpez.hpez_compress_async(gpu.handle, x.data_ptr(), shape, 0, 1e-3, None, out.data_ptr(),
                                 cap, sz.data_ptr(), st0.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    for seed in (12, 13):
        x.copy_(torch.from_numpy(fields.make("grf", shape, seed)).cuda())
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        size, status = sz.item(), st0.item()
        assert status == 0
        buf, ref = gpu.compress(x, 1e-3, 0)
        assert size == ref
        assert torch.equal(out[:size], buf[:ref])
    # decompress of one stream, replayed into a cleared output
    hdr = out[:512].cpu().numpy().tobytes()
    y = torch.empty_like(x)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    with torch.cuda.stream(cs):
        hpez.hpez_decompress_async(gpu.handle, out.data_ptr(), size, hdr, y.data_ptr(),
                                   y.numel(), st.data_ptr(), cs.cuda_stream)
    torch.cuda.synchronize()
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=cs):
        hpez.hpez_decompress_async(gpu.handle, out.data_ptr(), size, hdr, y.data_ptr(),
                                   y.numel(), st.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    want = gpu.decompress(out, size)
    for _ in range(2):
        y.fill_(float("nan"))
        st.fill_(-99)
        g2.replay()
        torch.cuda.synchronize()
        assert st.item() == 0 and torch.equal(y, want)
