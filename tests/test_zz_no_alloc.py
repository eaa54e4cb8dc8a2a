"""hpez_decompress_noalloc: decompression for callers that may not allocate
memory (an external memory manager owns the device heap, or a pre-sized
loop may not call cudaMalloc once running).  Its scratch is a fixed device
array inside the library; its output must equal hpez_decompress's, bit for
bit, on consecutive calls.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_12133_gb300 import build as B
    B.build()
    from paper_2311_12133_gb300 import hpez
    c = hpez.Context(0)
    yield c
    c.close()


def _noalloc(buf, size, shape):
    import torch
    from paper_2311_12133_gb300 import hpez
    out = torch.full(shape, float("nan"), dtype=torch.float32, device=buf.device)
    hpez.hpez_decompress_noalloc(buf.data_ptr(), size, out.data_ptr(), out.numel(),
                                 torch.cuda.current_stream().cuda_stream)
    return out


def test_noalloc_matches_decompress_twice(ctx):
    import torch
    from paper_2311_12133_gb300 import fields, hpez
    cases = [(fields.bumps((96, 80, 72), seed=3), {}),
             (fields.climate2d((300, 500), seed=1), {"same_level": 1}),
             (fields.grf((40000,), seed=2), {"interp": hpez.HPEZ_CUBIC_NAT})]
    for x, kw in cases:
        cfg = hpez.make_config(x.ndim, **kw)
        xd = torch.from_numpy(x).cuda()
        buf, size = ctx.compress(xd, 1e-3, hpez.HPEZ_EB_REL, cfg)
        ref = ctx.decompress(buf, size).cpu().numpy()
        for _ in range(2):  # the array keeps the last call's contents
            got = _noalloc(buf, size, x.shape).cpu().numpy()
            assert got.tobytes() == ref.tobytes()


def test_noalloc_matches_tuned_md_and_frozen_streams(ctx):
    """Streams of every sweep the decompressor can meet: auto-tuned ones
    (a block map, uniform or mixed), the multi-dimensional paradigm, a
    frozen dimension, and an explicit mixed block map."""
    import torch
    from paper_2311_12133_gb300 import fields, hpez
    cases = []
    for kind, shape, seed in (("grf", (64, 64, 64), 1), ("bumps", (70, 64, 40), 9),
                              ("aniso", (24, 96, 80), 2), ("climate2d", (400, 640), 3)):
        x = fields.make(kind, shape, seed)
        xd = torch.from_numpy(x).cuda()
        cap = hpez.hpez_compress_bound(x.shape)
        buf = torch.empty(cap, dtype=torch.uint8, device="cuda")
        size = hpez.hpez_compress_auto(ctx.handle, xd.data_ptr(), x.shape, hpez.HPEZ_EB_REL,
                                       1e-3, None, buf.data_ptr(), cap,
                                       torch.cuda.current_stream().cuda_stream)
        cases.append((x, buf, size))
    bm = np.random.default_rng(4).choice(np.array([0, 1, 2, 5, 6], np.uint8),
                                         size=hpez.hpez_blockmap_size((70, 64, 45), 32))
    for x, kw in ((fields.grf((50, 40, 64), seed=6), {"paradigm": 1, "interp": 2}),
                  (fields.grf((50, 40, 64), seed=7), {"paradigm": 1, "same_level": 1}),
                  (fields.aniso((12, 80, 96), seed=1), {"frozen_dim": 0}),
                  (fields.aniso((12, 80, 96), seed=2), {"frozen_dim": 0, "paradigm": 1}),
                  (fields.grf((70, 64, 45), seed=5), {"blockmap": bm})):
        xd = torch.from_numpy(x).cuda()
        buf, size = ctx.compress(xd, 1e-3, hpez.HPEZ_EB_REL, hpez.make_config(x.ndim, **kw))
        cases.append((x, buf, size))
    blockwise = 0
    for x, buf, size in cases:
        hdr = buf[:512].cpu().numpy().tobytes()
        blockwise += int.from_bytes(hdr[212:216], "little")
        ref = ctx.decompress(buf, size).cpu().numpy()
        for _ in range(2):
            got = _noalloc(buf, size, x.shape).cpu().numpy()
            assert got.tobytes() == ref.tobytes()
    assert blockwise >= 2  # block maps were among the streams


def test_noalloc_refuses_global_spline_streams(ctx):
    """A stream with a global natural-spline level is hpez_decompress's
    only."""
    import torch
    from paper_2311_12133_gb300 import fields, hpez
    x = torch.from_numpy(fields.grf((40, 40, 40), seed=8)).cuda()
    buf, size = ctx.compress(x, 1e-3, 1, hpez.make_config(3, interp=hpez.HPEZ_SPLINE_GLOBAL))
    out = torch.empty_like(x)
    with pytest.raises(hpez.HpezError) as e:
        hpez.hpez_decompress_noalloc(buf.data_ptr(), size, out.data_ptr(), out.numel(),
                                     torch.cuda.current_stream().cuda_stream)
    assert e.value.code == -8


def test_noalloc_refuses_fields_beyond_its_scratch(ctx):
    import torch
    from paper_2311_12133_gb300 import fields, hpez
    x = torch.from_numpy(fields.grf((130, 128, 128), seed=4)).cuda()
    assert x.numel() > hpez.HPEZ_NOALLOC_MAX_POINTS
    buf, size = ctx.compress(x, 1e-3)
    with pytest.raises(hpez.HpezError) as e:
        _noalloc(buf, size, tuple(x.shape))
    assert e.value.code == hpez.HPEZ_ERR_TOO_LARGE
    # a field at the limit still works afterwards
    y = torch.from_numpy(fields.grf((128, 128, 128), seed=5)).cuda()
    buf, size = ctx.compress(y, 1e-3)
    ref = ctx.decompress(buf, size)
    got = _noalloc(buf, size, tuple(y.shape))
    assert torch.equal(got, ref)


def test_noalloc_refuses_lorenzo_streams(ctx):
    """A Lorenzo-predictor stream (Sec. 6.5) is hpez_decompress's only."""
    import torch
    from paper_2311_12133_gb300 import hpez
    x = torch.rand((40, 40, 40), device="cuda")
    buf, size = ctx.compress(x, 1e-3, 1, hpez.make_config(3, predictor=1))
    out = torch.empty_like(x)
    with pytest.raises(hpez.HpezError) as e:
        hpez.hpez_decompress_noalloc(buf.data_ptr(), size, out.data_ptr(), out.numel(),
                                     torch.cuda.current_stream().cuda_stream)
    assert e.value.code == -8


def test_noalloc_refuses_lossless_streams(ctx):
    """A stream that went through the lossless stage is hpez_decompress's
    only (undoing the stage needs a buffer)."""
    import torch
    from paper_2311_12133_gb300 import fields, hpez
    x = torch.from_numpy(fields.bumps((40, 40, 40), seed=3)).cuda()
    buf, size = ctx.compress(x, 1e-1)
    z = torch.empty(size + 64, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    zs = hpez.hpez_lossless_encode(ctx.handle, buf.data_ptr(), size, z.data_ptr(), z.numel(),
                                   stream)
    assert zs < size
    out = torch.empty_like(x)
    with pytest.raises(hpez.HpezError) as e:
        hpez.hpez_decompress_noalloc(z.data_ptr(), zs, out.data_ptr(), out.numel(), stream)
    assert e.value.code == -8
    assert torch.equal(ctx.decompress(z, zs), ctx.decompress(buf, size))
