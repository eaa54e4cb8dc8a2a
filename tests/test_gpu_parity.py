"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

The bar is bit-exact: compressed bytes (codes, outliers, Huffman tables and
bitstream, header) and decompressed fields must equal the oracle's, a
floating-point tolerance of 0 ULP, because both sides perform the same IEEE
binary32 operations in the same order.
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


def _gpu_roundtrip(ctx, x, eb, mode, cfg=None):
    import torch
    from paper_2311_12133_gb300 import hpez
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    buf, size = ctx.compress(xd, eb, mode, cfg)
    stream = buf[:size].cpu().numpy().tobytes()
    y = ctx.decompress(buf, size).cpu().numpy()
    return stream, y


def _pair_configs(nd, **kw):
    from oracle import oracle as O
    from paper_2311_12133_gb300 import hpez
    return O.make_config(nd, **kw), hpez.make_config(nd, **kw)


def _check(ctx, oracle, x, eb=1e-3, mode=1, **kw):
    ocfg, gcfg = _pair_configs(x.ndim, **kw)
    want, st, _, recon = oracle.compress(x, eb, mode, ocfg, want_recon=True)
    got, y = _gpu_roundtrip(ctx, x, eb, mode, gcfg)
    assert len(got) == len(want), (len(got), len(want))
    if got != want:
        a = np.frombuffer(got, np.uint8)
        b = np.frombuffer(want, np.uint8)
        first = int(np.nonzero(a != b)[0][0])
        raise AssertionError(f"stream differs first at byte {first} of {len(want)}")
    assert y.tobytes() == oracle.decompress(want).tobytes()
    if not (mode == 1 and x.max() == x.min()):
        assert y.tobytes() == recon.tobytes()
        assert np.all(np.abs(y.astype(np.float64) - x) <= st.e)
    return st


def test_bumps_128_default(gpu, oracle):
    """The plain workload: 128^3 Gaussian bumps, rel eb 1e-3, cubic
    not-a-knot, fixed dimension order, no tuning."""
    from paper_2311_12133_gb300 import fields
    x = fields.bumps((128, 128, 128), seed=1)
    st = _check(gpu, oracle, x, 1e-3, 1)
    assert st.n_used > 2


@pytest.mark.parametrize("interp", [0, 1, 2])
@pytest.mark.parametrize("paradigm", [0, 1])
@pytest.mark.parametrize("same", [0, 1])
def test_interpolators_3d(gpu, oracle, interp, paradigm, same):
    from paper_2311_12133_gb300 import fields
    x = fields.grf((37, 50, 67), seed=interp * 4 + paradigm * 2 + same)
    _check(gpu, oracle, x, 1e-3, 1, interp=interp, paradigm=paradigm,
           same_level=same, anchor_stride=16)


@pytest.mark.parametrize("shape", [(1,), (2,), (5,), (1000,), (129,), (7, 5),
                                   (1, 300), (65, 129), (100, 3), (3, 4, 5),
                                   (1, 1, 77), (33, 1, 20), (17, 19, 23)])
def test_shapes_ragged(gpu, oracle, shape):
    rng = np.random.default_rng(len(shape) * 100 + shape[-1])
    x = rng.standard_normal(shape).cumsum(axis=-1).astype(np.float32)
    if x.size > 1 and x.max() == x.min():
        x.flat[0] += 1
    for A in (2, 8, 64):
        _check(gpu, oracle, x, 1e-2, 1, anchor_stride=A)
        _check(gpu, oracle, x, 0.05, 0, anchor_stride=A, interp=2, same_level=1)


@pytest.mark.parametrize("order", [(0, 1, 2), (2, 1, 0), (1, 2, 0), (2, 0, 1)])
def test_dim_orders(gpu, oracle, order):
    from paper_2311_12133_gb300 import fields
    x = fields.bumps((40, 33, 50), seed=7)
    _check(gpu, oracle, x, 1e-3, 1, order=order)
    # per-level orders and interpolators
    _check(gpu, oracle, x, 1e-4, 1, order=[order, (0, 1, 2), (1, 0, 2), order, order],
           interp=[2, 1, 0, 1, 2], same_level=[1, 0, 0, 1, 1], paradigm=[0, 1, 0, 1, 0])


@pytest.mark.parametrize("frozen", [0, 1, 2])
def test_frozen_dimension(gpu, oracle, frozen):
    from paper_2311_12133_gb300 import fields
    x = fields.aniso((12, 80, 96), seed=frozen)
    _check(gpu, oracle, x, 1e-3, 1, frozen_dim=frozen, paradigm=1,
           md_inv_var=(1.0, 3.0, 0.25))
    _check(gpu, oracle, x, 1e-3, 1, frozen_dim=frozen)


def test_alpha_beta_level_bounds(gpu, oracle):
    from paper_2311_12133_gb300 import fields
    x = fields.grf((64, 64, 64), seed=3)
    for a, b in ((1.5, 4.0), (2.0, 2.0), (1.25, 8.0)):
        _check(gpu, oracle, x, 1e-3, 1, alpha=a, beta=b)


def test_blockwise_map(gpu, oracle):
    from paper_2311_12133_gb300 import fields
    x = fields.grf((70, 64, 45), seed=5)
    rng = np.random.default_rng(9)
    nb = 3 * 2 * 2
    bm = rng.choice(np.array([0, 1, 2, 5, 6], np.uint8), size=nb)
    _check(gpu, oracle, x, 1e-3, 1, blockmap=bm)


def test_2d_and_1d_workloads(gpu, oracle):
    from paper_2311_12133_gb300 import fields
    x = fields.climate2d((180, 360), seed=2)
    _check(gpu, oracle, x, 1e-3, 1)
    _check(gpu, oracle, x, 1e-4, 1, paradigm=1, same_level=1, interp=2)
    y = fields.grf((5000,), seed=4)
    _check(gpu, oracle, y, 1e-3, 1)


def test_chunk_sizes_and_outliers(gpu, oracle):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((33, 40, 41)).astype(np.float32)
    for C in (256, 1024, 32768):
        _check(gpu, oracle, x, 1e-3, 1, chunk_syms=C)
    # white noise with a tiny bound: many outliers and a wide alphabet
    st = _check(gpu, oracle, x, 1e-6, 1)
    assert st.n_outliers > 0
    # alphabet larger than the shared-memory codebook (global-memory path)
    st = _check(gpu, oracle, x, 2e-5, 1)
    assert st.n_used > 8192


def test_degenerate_fields(gpu, oracle):
    c = np.full((20, 30), 1.25, np.float32)
    _check(gpu, oracle, c, 1e-3, 1)  # constant: header-only stream
    _check(gpu, oracle, c, 1e-3, 0)  # absolute bound: a regular stream
    one = np.array([3.5], np.float32)
    _check(gpu, oracle, one, 0.1, 0)
    # a linear ramp on a grid that ends on anchor lines: every code is the
    # zero-error code, so the code table has a single symbol
    lin = np.arange(17 * 257, dtype=np.float32).reshape(17, 257)
    st = _check(gpu, oracle, lin, 0.25, 0, anchor_stride=16)
    assert st.n_used == 1


def test_error_codes(gpu):
    import torch
    from paper_2311_12133_gb300 import hpez
    x = torch.zeros(1000, device="cuda")
    x[5] = float("nan")
    with pytest.raises(hpez.HpezError) as e:
        gpu.compress(x, 1e-3, hpez.HPEZ_EB_REL)
    assert e.value.code == -2
    x = torch.randn(64, 64, device="cuda")
    out = torch.empty(600, dtype=torch.uint8, device="cuda")
    with pytest.raises(hpez.HpezError) as e:
        hpez.hpez_compress(gpu.handle, x.data_ptr(), (64, 64), 1, 1e-3, None,
                           out.data_ptr(), 600, 0)
    assert e.value.code == -3
    buf, size = gpu.compress(x, 1e-3)
    bad = buf.clone()
    bad[0] ^= 0xFF
    with pytest.raises(hpez.HpezError):
        gpu.decompress(bad, size, shape=(64, 64))
    with pytest.raises(hpez.HpezError):
        gpu.decompress(buf, 300, shape=(64, 64))


def test_host_buffer_entry_points(gpu, oracle):
    from paper_2311_12133_gb300 import fields, hpez
    x = fields.bumps((30, 40, 50), seed=2)
    out = np.zeros(hpez.hpez_compress_bound(x.shape), np.uint8)
    size = hpez.hpez_compress_host(gpu.handle, x, 1, 1e-3, None, out)
    want, _, _, recon = oracle.compress(x, 1e-3, 1, want_recon=True)
    assert out[:size].tobytes() == want
    y = np.zeros(x.size, np.float32)
    hpez.hpez_decompress_host(gpu.handle, out, size, y)
    assert y.tobytes() == recon.tobytes()


def test_determinism_repeated(gpu):
    import torch
    from paper_2311_12133_gb300 import fields
    x = torch.from_numpy(fields.lognormal((64, 64, 64), seed=1)).cuda()
    ref = None
    for _ in range(5):
        buf, size = gpu.compress(x, 1e-4)
        b = buf[:size].cpu().numpy().tobytes()
        ref = ref or b
        assert b == ref


@pytest.fixture
def opts(gpu):
    """Restore the context's execution options after a test."""
    from paper_2311_12133_gb300 import hpez
    yield gpu
    hpez.hpez_set_option(gpu.handle, hpez.HPEZ_OPT_FUSED_LEVELS, 1)
    hpez.hpez_set_option(gpu.handle, hpez.HPEZ_OPT_STREAM_LEVELS, 1)
    hpez.hpez_set_option(gpu.handle, hpez.HPEZ_OPT_DROP_COPY, 0)
    hpez.hpez_set_option(gpu.handle, hpez.HPEZ_OPT_WARP_LEVELS, 1)
    hpez.hpez_set_option(gpu.handle, hpez.HPEZ_OPT_STREAM_CHUNKS, 0)
    for o in (hpez.HPEZ_OPT_TILE_E0, hpez.HPEZ_OPT_TILE_E1, hpez.HPEZ_OPT_TILE_E2):
        hpez.hpez_set_option(gpu.handle, o, 0)


@pytest.mark.parametrize("tile", [(2, 4, 8), (2, 2, 2), (4, 6, 10), (6, 2, 4)])
@pytest.mark.parametrize("order,same,interp", [((0, 1, 2), 0, 1), ((2, 1, 0), 1, 1),
                                               ((1, 0, 2), 1, 2), ((0, 2, 1), 0, 0)])
def test_fused_level_tiles(opts, oracle, tile, order, same, interp):
    """Small tiles make most of every tile halo: the recomputed halo points
    must equal the neighbouring tiles' own results bit for bit."""
    from paper_2311_12133_gb300 import fields, hpez
    for o, e in zip((hpez.HPEZ_OPT_TILE_E0, hpez.HPEZ_OPT_TILE_E1, hpez.HPEZ_OPT_TILE_E2), tile):
        hpez.hpez_set_option(opts.handle, o, e)
    x = fields.grf((29, 36, 43), seed=sum(tile) + same)
    _check(opts, oracle, x, 1e-3, 1, order=order, same_level=same, interp=interp,
           anchor_stride=16)


def test_fused_tiles_blockwise_frozen_2d(opts, oracle):
    from paper_2311_12133_gb300 import fields, hpez
    hpez.hpez_set_option(opts.handle, hpez.HPEZ_OPT_TILE_E1, 4)
    hpez.hpez_set_option(opts.handle, hpez.HPEZ_OPT_TILE_E2, 6)
    x = fields.grf((70, 64, 45), seed=5)
    bm = np.random.default_rng(3).choice(np.array([0, 1, 2, 5, 6], np.uint8), size=12)
    _check(opts, oracle, x, 1e-3, 1, blockmap=bm, order=(1, 2, 0))
    y = fields.aniso((10, 50, 60), seed=1)
    _check(opts, oracle, y, 1e-3, 1, frozen_dim=0, same_level=1)
    z = fields.climate2d((90, 150), seed=4)
    _check(opts, oracle, z, 1e-3, 1, same_level=1, order=(1, 0))


def test_per_pass_path_still_exact(opts, oracle):
    """The one-kernel-per-pass path (used for multi-dimensional levels)
    forced on for 1D-style levels too."""
    from paper_2311_12133_gb300 import fields, hpez
    hpez.hpez_set_option(opts.handle, hpez.HPEZ_OPT_FUSED_LEVELS, 0)
    x = fields.grf((40, 41, 42), seed=8)
    _check(opts, oracle, x, 1e-3, 1)
    _check(opts, oracle, x, 1e-3, 1, same_level=1, interp=2, order=(2, 0, 1))


@pytest.mark.parametrize("shape,frozen", [((37, 50, 67), -1), ((129, 257), -1),
                                          ((40, 36, 44), 1), ((3000,), -1)])
@pytest.mark.parametrize("interp,same", [(0, 0), (1, 0), (2, 0), (0, 1)])
def test_md_levels(gpu, oracle, shape, frozen, interp, same):
    """Multi-dimensional levels (one launch per sub-pass) in 1D, 2D, 3D and
    with a frozen dimension."""
    from paper_2311_12133_gb300 import fields
    if len(shape) == 1:
        x = np.cumsum(np.random.default_rng(5).normal(0, 1, shape[0])).astype(np.float32)
    else:
        x = fields.grf(shape, seed=len(shape) * 10 + interp)
    _check(gpu, oracle, x, 1e-3, 1, interp=interp, paradigm=1, same_level=same,
           frozen_dim=frozen, md_inv_var=(1.0, 2.5, 0.7))


@pytest.mark.parametrize("shape,eb", [((40, 48, 64), 1e-3), ((33, 17, 128), 1e-3),
                                      ((9, 70, 136), 1e-4), ((64, 40, 256), 1e-3),
                                      ((2, 3, 8), 1e-3), ((5, 16, 24), 1e-6),
                                      ((66, 20, 16), 1e-3)])
@pytest.mark.parametrize("interp", [0, 1, 2])
def test_md_stream_level(opts, oracle, shape, eb, interp):
    """The finest 3D multi-dimensional level streamed in one launch (rows a
    multiple of 8 points; compress also needs the coarse rows in whole
    16-byte units, i.e. rows a multiple of 16): partial row and column
    tiles, odd and even plane counts, chunk boundaries, outliers (eb 1e-6);
    equal to the oracle, and to the two-launch path, which needs one launch
    more."""
    import torch
    from paper_2311_12133_gb300 import fields, hpez
    hpez.hpez_set_option(opts.handle, hpez.HPEZ_OPT_WARP_LEVELS, 0)
    x = fields.grf(shape, seed=sum(shape) + interp)
    kw = dict(interp=interp, paradigm=1, md_inv_var=(1.0, 2.5, 0.7))
    _check(opts, oracle, x, eb, 1, **kw)
    _, gcfg = _pair_configs(3, **kw)
    xd = torch.from_numpy(x).cuda()
    count = lambda: hpez.hpez_launch_count(opts.handle)
    runs = {}
    for on in (1, 0):
        hpez.hpez_set_option(opts.handle, hpez.HPEZ_OPT_STREAM_LEVELS, on)
        n0 = count()
        buf, size = opts.compress(xd, eb, 1, gcfg)
        n1 = count()
        y = opts.decompress(buf, size).cpu().numpy()
        runs[on] = (buf[:size].cpu().numpy().tobytes(), y.tobytes(), n1 - n0, count() - n1)
    assert runs[1][0] == runs[0][0] and runs[1][1] == runs[0][1]
    assert runs[0][2] - runs[1][2] == (1 if shape[2] % 16 == 0 else 0)
    assert runs[0][3] - runs[1][3] == 1


def test_bounded_wait_expires(opts, oracle):
    """A copy that never lands makes its bounded wait expire: the first CTA of
    the streamed level kernel leaves out one plane's copies on request, the
    call returns HPEZ_ERR_TIMEOUT within seconds, and the next call on the
    same context is exact again (compress and decompress)."""
    import time
    import torch
    from paper_2311_12133_gb300 import fields, hpez
    hpez.hpez_set_option(opts.handle, hpez.HPEZ_OPT_WARP_LEVELS, 0)
    x = fields.grf((40, 48, 64), seed=3)
    kw = dict(interp=0, paradigm=1)
    _, gcfg = _pair_configs(3, **kw)
    xd = torch.from_numpy(x).cuda()
    buf, size = opts.compress(xd, 1e-3, 1, gcfg)
    for item in (1, 3):
        hpez.hpez_set_option(opts.handle, hpez.HPEZ_OPT_DROP_COPY, item)
        t0 = time.time()
        with pytest.raises(hpez.HpezError) as e:
            opts.compress(xd, 1e-3, 1, gcfg)
        assert e.value.code == -9
        with pytest.raises(hpez.HpezError) as e:
            opts.decompress(buf, size)
        assert e.value.code == -9
        assert time.time() - t0 < 60
    hpez.hpez_set_option(opts.handle, hpez.HPEZ_OPT_DROP_COPY, 0)
    _check(opts, oracle, x, 1e-3, 1, **kw)


@pytest.mark.parametrize("code", [0, 1, 2, 5, 6])
@pytest.mark.parametrize("paradigm", [0, 1])
def test_uniform_blockmap(gpu, oracle, code, paradigm):
    """A block map with one code everywhere runs as that interpolator."""
    from paper_2311_12133_gb300 import fields, hpez
    shape = (48, 40, 36)
    x = fields.bumps(shape, seed=code)
    nb = hpez.hpez_blockmap_size(shape, 16)
    _check(gpu, oracle, x, 1e-3, 1, blockmap=np.full(nb, code, np.uint8),
           block_size=16, paradigm=paradigm)


@pytest.mark.parametrize("shape", [(48, 64, 256), (49, 40, 128), (50, 17, 144), (9, 70, 136),
                                   (5, 16, 24), (66, 20, 16), (2, 3, 8), (37, 50, 68),
                                   (3, 5, 6), (7, 33, 130), (16, 18, 4), (20, 19, 62),
                                   (11, 2, 120), (30, 50, 500)])
@pytest.mark.parametrize("interp", [0, 1, 2])
@pytest.mark.parametrize("chunks", [0, 1, 3])
def test_md_warp_level(opts, oracle, shape, interp, chunks):
    """The finest 3D multi-dimensional level with one warp per strip
    (rows of an even number of points): partial row and column strips, the
    column strips' halo lanes, short last strips that extrapolate, odd and
    even plane counts, chunks of planes (one chunk walks every plane);
    equal to the oracle, and the kernel taken (one launch for the level, two
    without it)."""
    import torch
    from paper_2311_12133_gb300 import fields, hpez
    hpez.hpez_set_option(opts.handle, hpez.HPEZ_OPT_STREAM_CHUNKS, chunks)
    x = fields.grf(shape, seed=sum(shape) + 3 * interp + chunks)
    kw = dict(interp=interp, paradigm=1, md_inv_var=(1.0, 2.5, 0.7))
    n0 = hpez.hpez_launch_count(opts.handle)
    _check(opts, oracle, x, 1e-3, 1, **kw)
    n_warp = hpez.hpez_launch_count(opts.handle) - n0
    for o in (hpez.HPEZ_OPT_WARP_LEVELS, hpez.HPEZ_OPT_STREAM_LEVELS):
        hpez.hpez_set_option(opts.handle, o, 0)
    n0 = hpez.hpez_launch_count(opts.handle)
    _check(opts, oracle, x, 1e-3, 1, **kw)
    assert hpez.hpez_launch_count(opts.handle) - n0 >= n_warp + 2
    hpez.hpez_set_option(opts.handle, hpez.HPEZ_OPT_WARP_LEVELS, 1)
    # escapes inside the strips
    _check(opts, oracle, fields.make("lognormal", shape, 2), 1e-6, 1, **kw)
