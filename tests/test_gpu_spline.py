"""Parity of the CUDA global natural-spline interpolator (interp 3: the
natural cubic spline through every known point of a pass line, solved per
line) with the oracle.  Bit-exact: both sides run the Thomas algorithm and
the midpoint form in binary32 in the same order."""
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


def _check(ctx, oracle, x, eb, mode, **kw):
    import torch
    from paper_2311_12133_gb300 import hpez
    ocfg = oracle.make_config(x.ndim, **kw)
    gcfg = hpez.make_config(x.ndim, **kw)
    want, st, _, recon = oracle.compress(x, eb, mode, ocfg, want_recon=True)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    buf, size = ctx.compress(xd, eb, mode, gcfg)
    got = buf[:size].cpu().numpy().tobytes()
    assert len(got) == len(want), (len(got), len(want))
    if got != want:
        a = np.frombuffer(got, np.uint8)
        b = np.frombuffer(want, np.uint8)
        first = int(np.nonzero(a != b)[0][0])
        raise AssertionError(f"stream differs first at byte {first} of {len(want)}")
    y = ctx.decompress(buf, size).cpu().numpy()
    assert y.tobytes() == oracle.decompress(want).tobytes()
    if x.max() != x.min():
        assert y.tobytes() == recon.tobytes()
        assert np.all(np.abs(y.astype(np.float64) - x) <= st.e)
    return st


@pytest.mark.parametrize("shape,A,order", [
    ((37, 50, 67), None, (0, 1, 2)),
    ((64, 64, 64), 16, (2, 0, 1)),
    ((33, 9, 70), 8, (1, 2, 0)),
    ((129, 257), None, (0, 1)),
    ((96, 200), 32, (1, 0)),
    ((5000,), None, (0,)),
    ((6,), 4, (0,)),
    ((3, 4, 5), 2, (0, 1, 2)),
])
def test_spline_fields(gpu, oracle, shape, A, order):
    from paper_2311_12133_gb300 import fields
    x = fields.grf(shape, seed=len(shape) + sum(shape))
    kw = dict(interp=3, order=order)
    if A is not None:
        kw["anchor_stride"] = A
    _check(gpu, oracle, x, 1e-3, 1, **kw)


def test_spline_mixed_levels_frozen_and_escapes(gpu, oracle):
    """Spline on some levels, local interpolators on others; a frozen
    dimension; a tight bound on a heavy-tailed field for many escapes
    (the level-1 decompressor's scratch keeps them intact)."""
    from paper_2311_12133_gb300 import fields
    x = fields.grf((40, 36, 50), seed=2)
    _check(gpu, oracle, x, 1e-3, 1, interp=[3, 1, 3, 0, 3], frozen_dim=1)
    y = fields.make("lognormal", (40, 48, 64), seed=5)
    st = _check(gpu, oracle, y, 1e-6, 1, interp=3, chunk_syms=4096)
    assert st.n_outliers > 100
    i, j, k = np.indices((29, 34, 40))
    lin = (3 * i - 2 * j + 5 * k + 7).astype(np.float32)
    _check(gpu, oracle, lin, 0.01, 0, interp=3, anchor_stride=8)


def test_spline_refused_forms(gpu):
    import torch
    from paper_2311_12133_gb300 import hpez
    x = torch.rand((40, 40, 40), device="cuda")
    for kw in (dict(paradigm=1), dict(same_level=1)):
        with pytest.raises(hpez.HpezError) as e:
            gpu.compress(x, 1e-3, 1, hpez.make_config(3, interp=3, **kw))
        assert e.value.code == -1
    cfg = hpez.make_config(3, interp=3)
    with pytest.raises(hpez.HpezError) as e:
        hpez.Batch(gpu, fields=[(x, 1e-3, 1, cfg)])
    assert e.value.code == -8
    buf, size = gpu.compress(x, 1e-3, 1, cfg)
    out = torch.empty_like(x)
    with pytest.raises(hpez.HpezError) as e:
        hpez.hpez_decompress_noalloc(buf.data_ptr(), size, out.data_ptr(), out.numel(),
                                     torch.cuda.current_stream().cuda_stream)
    assert e.value.code == -8
