"""Parity of the CUDA Lorenzo predictor (Sec. 6.5; block-local on blocks of
side A, neighbours outside the block read 0) with the oracle, and of the
tuner's choice between it and interpolation.

The bar is bit-exact, as for interpolation: the compressed bytes and the
decompressed field equal the oracle's, because both sides evaluate the
stencil's terms in the same order in binary32 with the same quantizer.
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


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("shape,A", [
    ((37, 50, 67), None),      # ragged blocks of side 32 on every axis
    ((64, 64, 64), 16),        # whole blocks, 64 of them
    ((33, 9, 70), 8),          # side-1 tails
    ((20, 21, 22), 4),         # blocks shorter than an input segment
    ((9, 10, 11), 2),
    ((70, 45, 96), None),      # rows of 16-byte segments, ragged in i0 and i1
    ((129, 257), None),        # 2D, ragged blocks of side 64
    ((96, 200), 64),           # 2D, rows of 16-byte segments
    ((300, 41), 128),          # 2D, one CTA column per block row
    ((5000,), None),           # 1D
    ((5,), 8),                 # 1D, one partial block
])
def test_lorenzo_fields(gpu, oracle, order, shape, A):
    from paper_2311_12133_gb300 import fields
    x = fields.grf(shape, seed=len(shape) * 10 + order)
    kw = dict(predictor=order)
    if A is not None:
        kw["anchor_stride"] = A
    _check(gpu, oracle, x, 1e-3, 1, **kw)


@pytest.mark.parametrize("order", [1, 2])
def test_lorenzo_outliers_and_chunks(gpu, oracle, order):
    """A heavy-tailed field at a tight bound: many escapes (code 0) whose
    values the decompressor reads from the outlier list mid-recurrence."""
    from paper_2311_12133_gb300 import fields
    x = fields.make("lognormal", (40, 48, 64), seed=5)
    st = _check(gpu, oracle, x, 1e-6, 1, predictor=order, chunk_syms=4096)
    assert st.n_outliers > 100


def test_lorenzo_integer_exact(gpu, oracle):
    """Integers at e = 1/2: every code is exact, both orders."""
    rng = np.random.default_rng(3)
    g = rng.integers(-50, 50, size=(40, 40))
    h = rng.integers(-50, 50, size=(40, 40))
    x = (g[:, :, None] + h[None, :, :]).astype(np.float32)
    for order in (1, 2):
        _check(gpu, oracle, x, 0.5, 0, predictor=order)


def test_lorenzo_frozen_and_constant(gpu, oracle):
    from paper_2311_12133_gb300 import fields
    x = fields.grf((30, 40, 50), seed=4)
    _check(gpu, oracle, x, 1e-3, 1, predictor=1, frozen_dim=1)
    c = np.full((20, 30, 40), 2.5, np.float32)
    _check(gpu, oracle, c, 1e-3, 1, predictor=2)


def test_lorenzo_unsupported_forms(gpu):
    """Blocks whose columns do not fit a CTA and a block-wise map with the
    Lorenzo predictor are refused; the batched and served forms take the
    Lorenzo predictor with the same results as the single call."""
    import torch
    from paper_2311_12133_gb300 import hpez
    x = torch.rand((70, 70, 70), device="cuda")
    with pytest.raises(hpez.HpezError) as e:
        gpu.compress(x, 1e-3, 1, hpez.make_config(3, predictor=1, anchor_stride=64))
    assert e.value.code == -8
    bm = np.zeros(hpez.hpez_blockmap_size((70, 70, 70), 32), np.uint8)
    with pytest.raises(hpez.HpezError) as e:
        gpu.compress(x, 1e-3, 1, hpez.make_config(3, predictor=1, blockmap=bm))
    assert e.value.code == -1
    cfg = hpez.make_config(3, predictor=1)
    cfg.predictor = 3
    with pytest.raises(hpez.HpezError) as e:
        gpu.compress(x, 1e-3, 1, cfg)
    assert e.value.code == -1
    with pytest.raises(hpez.HpezError) as e:
        hpez.Batch(gpu, fields=[(x, 1e-3, 1, hpez.make_config(3, predictor=1,
                                                              anchor_stride=64))])
    assert e.value.code == -8
    # a Lorenzo field through the served form: the stream and the field of
    # the single call (the no-allocation decompressor refuses the stream,
    # tested with it)
    small = torch.rand((40, 40, 40), device="cuda")
    cfg2 = hpez.make_config(3, predictor=2)
    buf, size = gpu.compress(small, 1e-3, 1, cfg2)
    want = buf[:size].cpu().numpy()
    y = gpu.decompress(buf, size)
    srv = hpez.Server(gpu, 1 << 28, 4)
    rc, hc = srv.submit_compress(small.cpu().numpy(), 1e-3, 1, cfg2)
    rd, hd = srv.submit_decompress(want.copy(), size)
    done = {}
    for _ in range(10000):
        srv.step()
        for rid, st, sz, _ in srv.poll():
            done[rid] = (st, sz)
        if len(done) == 2:
            break
    srv.close()
    assert done[rc] == (0, size) and done[rd][0] == 0
    assert hc[:size].tobytes() == want.tobytes()
    assert hd.tobytes() == y.cpu().numpy().tobytes()
    assert (y - small).abs().max().item() <= 1e-3 * (small.max() - small.min()).item()


def _lorenzo_field():
    rng = np.random.default_rng(1)
    n = (64, 64, 64)
    g = rng.normal(0, 1, (n[0], n[1]))
    h = rng.normal(0, 1, (n[1], n[2]))
    return (g[:, :, None] + h[None, :, :]).astype(np.float32)


def test_tune_selects_lorenzo(gpu, oracle):
    """On a field without triple coupling the GPU tuner, like the oracle's,
    selects the Lorenzo predictor; the tuned stream equals the oracle's."""
    import torch
    from paper_2311_12133_gb300 import hpez
    x = _lorenzo_field()
    xd = torch.from_numpy(x).cuda()
    g_cfg, g_rep = gpu.tune(xd, 1e-3, 1)
    o_cfg, o_rep = oracle.tune(x, 1e-3, oracle.EB_REL)
    assert o_rep.lorenzo_better == 1 and o_cfg.predictor in (1, 2)
    assert g_rep.lorenzo_better == o_rep.lorenzo_better
    assert list(g_rep.lorenzo_bits) == list(o_rep.lorenzo_bits)
    assert g_cfg.predictor == o_cfg.predictor and g_cfg.blockwise == 0
    buf, size = gpu.compress(xd, 1e-3, 1, g_cfg)
    want, _, _, _ = oracle.compress(x, 1e-3, oracle.EB_REL, o_cfg)
    assert buf[:size].cpu().numpy().tobytes() == want
    # the one-call form takes the same path
    cap = hpez.hpez_compress_bound(x.shape)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    n = hpez.hpez_compress_auto(gpu.handle, xd.data_ptr(), x.shape, 1, 1e-3, None,
                                out.data_ptr(), cap)
    assert out[:n].cpu().numpy().tobytes() == want
    # a large coefficient keeps interpolation on both sides
    g2, r2 = gpu.tune(xd, 1e-3, 1, hpez.hpez_default_tune_params(lorenzo_coef=1e6))
    o2, q2 = oracle.tune(x, 1e-3, oracle.EB_REL, oracle.default_tune_params(lorenzo_coef=1e6))
    assert g2.predictor == o2.predictor == 0 and r2.lorenzo_better == q2.lorenzo_better == 0


def test_lorenzo_bounded_wait_expires(gpu, oracle):
    """The box-fed Lorenzo kernel's waits are bounded: on request the first
    warp of the first CTA leaves out one box (the prologue's, or a later
    one), its wait expires, compress and decompress return HPEZ_ERR_TIMEOUT
    within seconds, and the next calls on the context are exact."""
    import time
    import torch
    from paper_2311_12133_gb300 import fields, hpez
    x = fields.grf((64, 64, 64), seed=8)
    xd = torch.from_numpy(x).cuda()
    cfg = hpez.make_config(3, predictor=1)
    buf, size = gpu.compress(xd, 1e-3, 1, cfg)
    try:
        for item in (1, 3):
            hpez.hpez_set_option(gpu.handle, hpez.HPEZ_OPT_DROP_COPY, item)
            t0 = time.time()
            with pytest.raises(hpez.HpezError) as e:
                gpu.compress(xd, 1e-3, 1, cfg)
            assert e.value.code == -9
            with pytest.raises(hpez.HpezError) as e:
                gpu.decompress(buf, size)
            assert e.value.code == -9
            assert time.time() - t0 < 60
    finally:
        hpez.hpez_set_option(gpu.handle, hpez.HPEZ_OPT_DROP_COPY, 0)
    _check(gpu, oracle, x, 1e-3, 1, predictor=1)

