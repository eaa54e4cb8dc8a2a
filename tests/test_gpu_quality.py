"""Parity of the quality-metric target (Eq. 1 with M = PSNR) and of the
integer inputs with the oracle, through the C-ABI.

The PSNR's squared errors are an exact integer sum, so the metric, every
decision of the bound search, the bound found, the stream and the
reconstruction equal the oracle's bit for bit; the integer streams and the
rounded integers likewise.
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


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def test_psnr_metric(gpu, oracle):
    import torch
    from paper_2311_12133_gb300 import fields, hpez
    x = fields.grf((50, 60, 70), seed=2)
    e = np.float32(1e-3 * float(x.max() - x.min()))
    y = (x + np.random.default_rng(3).uniform(-e, e, x.shape)).astype(np.float32)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    for unit in (float(e) / 65536, float(e) / 1024):
        got = hpez.hpez_psnr(gpu.handle, xd.data_ptr(), yd.data_ptr(), x.size, unit, _stream())
        assert got == oracle.psnr(x, y, unit)
    assert hpez.hpez_psnr(gpu.handle, xd.data_ptr(), xd.data_ptr(), x.size, 1.0,
                          _stream())[0] == float("inf")
    bad = x.copy()
    bad[1, 2, 3] = np.inf
    with pytest.raises(hpez.HpezError) as err:
        hpez.hpez_psnr(gpu.handle, torch.from_numpy(bad).cuda().data_ptr(), yd.data_ptr(),
                       x.size, float(e) / 65536, _stream())
    assert err.value.code == -2


@pytest.mark.parametrize("kind,shape,target", [("grf", (24, 28, 32), 60.0),
                                               ("bumps", (30, 26, 20), 80.0),
                                               ("climate2d", (60, 90), 70.0),
                                               ("lognormal", (40, 44, 48), 90.0)])
def test_psnr_target_equals_oracle(gpu, oracle, kind, shape, target):
    import torch
    from paper_2311_12133_gb300 import fields, hpez
    x = fields.make(kind, shape, 5)
    want, we, wp = oracle.compress_psnr(x, target)
    xd = torch.from_numpy(x).cuda()
    cap = hpez.hpez_compress_bound(shape)
    buf = torch.empty(cap, dtype=torch.uint8, device="cuda")
    size, e, p = hpez.hpez_compress_psnr(gpu.handle, xd.data_ptr(), shape, target, None,
                                         buf.data_ptr(), cap, _stream())
    assert (e, p) == (we, wp)
    assert buf[:size].cpu().numpy().tobytes() == want
    assert p >= target
    y = gpu.decompress(buf, size).cpu().numpy()
    assert y.tobytes() == oracle.decompress(want).tobytes()


@pytest.mark.parametrize("dtype", ["int16", "uint16", "int32"])
@pytest.mark.parametrize("eb,mode,tune", [(0.4, 0, False), (3.0, 0, False), (1e-3, 1, True)])
def test_integer_fields_equal_oracle(gpu, oracle, dtype, eb, mode, tune):
    """A 2D image and a 3D movie of integers (the shapes of the paper's
    integer datasets, synthetic), lossless and lossy, plain and tuned."""
    import torch
    from paper_2311_12133_gb300 import fields, hpez
    dt = np.dtype(dtype)
    code = {"int16": hpez.HPEZ_DTYPE_I16, "uint16": hpez.HPEZ_DTYPE_U16,
            "int32": hpez.HPEZ_DTYPE_I32}[dtype]
    scale, off = {"int16": (8000, 0), "uint16": (15000, 32000), "int32": (2e6, 1e5)}[dtype]
    for x0 in (fields.climate2d((120, 170), seed=1), fields.bumps((16, 48, 64), seed=2)):
        x = np.clip(np.rint((x0 - x0.mean()) / (x0.std() + 1e-9) * scale / 4 + off),
                    np.iinfo(dt).min, np.iinfo(dt).max).astype(dt)
        want = oracle.compress_typed(x, eb, mode, tune=tune)
        # uint16 travels through torch as int16 storage (same bytes)
        store = np.int32 if dtype == "int32" else np.int16
        xd = torch.from_numpy(x.view(store)).cuda()
        cap = hpez.hpez_compress_bound(x.shape)
        buf = torch.empty(cap, dtype=torch.uint8, device="cuda")
        size = hpez.hpez_compress_typed(gpu.handle, xd.data_ptr(), code, x.shape, mode, eb,
                                        None, tune, None, buf.data_ptr(), cap, _stream())
        assert buf[:size].cpu().numpy().tobytes() == want
        out = torch.empty(x.shape, dtype=torch.int32 if dtype == "int32" else torch.int16,
                          device="cuda")
        hpez.hpez_decompress_typed(gpu.handle, buf.data_ptr(), size, out.data_ptr(), code,
                                   x.size, _stream())
        y = out.cpu().numpy().view(dt)
        assert y.tobytes() == oracle.decompress_typed(want, dt).tobytes()
        if eb < 1 and mode == 0:
            assert np.array_equal(y, x)


def test_integer_refusals(gpu):
    import torch
    from paper_2311_12133_gb300 import hpez
    x = torch.tensor([[0, 1 << 25]], dtype=torch.int32, device="cuda")
    buf = torch.empty(hpez.hpez_compress_bound((1, 2)), dtype=torch.uint8, device="cuda")
    with pytest.raises(hpez.HpezError):
        hpez.hpez_compress_typed(gpu.handle, x.data_ptr(), hpez.HPEZ_DTYPE_I32, (1, 2), 0, 1.0,
                                 None, False, None, buf.data_ptr(), buf.numel(), _stream())
    y = torch.arange(100, dtype=torch.int16, device="cuda").reshape(10, 10)
    buf = torch.empty(hpez.hpez_compress_bound((10, 10)), dtype=torch.uint8, device="cuda")
    size = hpez.hpez_compress_typed(gpu.handle, y.data_ptr(), hpez.HPEZ_DTYPE_I16, (10, 10), 0,
                                    1.0, None, False, None, buf.data_ptr(), buf.numel(),
                                    _stream())
    out = torch.empty((10, 10), dtype=torch.int16, device="cuda")
    with pytest.raises(hpez.HpezError):
        hpez.hpez_decompress_typed(gpu.handle, buf.data_ptr(), size, out.data_ptr(),
                                   hpez.HPEZ_DTYPE_U16, 100, _stream())
