"""Parity of the CUDA auto-tuner (hpez_tune, through the C-ABI) with the
oracle's tuner (Sec. 6).

The bar is exact: every tuned field of theta, the block map and every
intermediate result of the report equal the oracle's, because all scores
are integers computed from bit-identical binary32 predictions.  A tuned
theta then compresses to the oracle's bytes.
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


REPORT_FIELDS = ("stats_count", "mse_lin", "mse_cub", "nonsmooth_dim", "froze",
                 "lorenzo_better", "n_sample_blocks", "bits", "lorenzo_bits",
                 "level_choice", "level_score")


def _val(v):
    try:
        return [_val(e) for e in v]
    except TypeError:
        return v


def _compare(g_cfg, g_rep, o_cfg, o_rep):
    for f in ("anchor_stride", "frozen_dim", "chunk_syms", "blockwise",
              "block_size", "predictor", "alpha", "beta"):
        assert getattr(g_cfg, f) == getattr(o_cfg, f), f
    for f in ("md_inv_var", "interp", "paradigm", "same_level", "order"):
        assert _val(getattr(g_cfg, f)) == _val(getattr(o_cfg, f)), f
    for f in REPORT_FIELDS:
        assert _val(getattr(g_rep, f)) == _val(getattr(o_rep, f)), f
    if o_cfg.blockwise:
        assert np.array_equal(g_cfg._blockmap_ref, o_cfg._blockmap_ref)


def _params(mod, **kw):
    if mod.__name__.endswith("oracle"):
        return mod.default_tune_params(**kw)
    return mod.hpez_default_tune_params(**kw)


def _tune_both(ctx, oracle, x, eb, mode, **kw):
    import torch
    from paper_2311_12133_gb300 import hpez
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    g_cfg, g_rep = ctx.tune(xd, eb, mode, _params(hpez, **kw))
    o_cfg, o_rep = oracle.tune(x, eb, mode, _params(oracle, **kw))
    _compare(g_cfg, g_rep, o_cfg, o_rep)
    return xd, g_cfg, o_cfg, o_rep


def _compress_equal(ctx, oracle, xd, x, eb, mode, g_cfg, o_cfg):
    buf, size = ctx.compress(xd, eb, mode, g_cfg)
    got = buf[:size].cpu().numpy().tobytes()
    want, st, _, _ = oracle.compress(x, eb, mode, o_cfg)
    assert got == want
    y = ctx.decompress(buf, size).cpu().numpy()
    assert np.all(np.abs(y.astype(np.float64) - x) <= st.e)


@pytest.mark.parametrize("kind,shape,eb", [
    ("grf", (65, 65, 65), 1e-3),
    ("bumps", (96, 80, 72), 1e-3),
    ("grf", (40, 52, 33), 1e-2),
    ("lognormal", (64, 48, 70), 1e-4),
    ("climate2d", (129, 257), 1e-3),
    ("grf", (200, 150), 1e-2),
])
def test_tune_matches_oracle(gpu, oracle, kind, shape, eb):
    from paper_2311_12133_gb300 import fields
    x = fields.make(kind, shape, seed=21)
    xd, g_cfg, o_cfg, _ = _tune_both(gpu, oracle, x, eb, 1)
    _compress_equal(gpu, oracle, xd, x, eb, 1, g_cfg, o_cfg)


@pytest.mark.parametrize("kw", [
    dict(anchor_stride=8, block_rate=0.1),
    dict(anchor_stride=16, allow_natural=0),
    dict(anchor_stride=8, allow_same_level=0, block_size=16),
    dict(tune_levels=0, tune_eb=0),
    dict(tune_freeze=0, tune_blockwise=0, sample_rate=0.01),
    dict(anchor_stride=4, block_rate=0.05, sub_frac=0.1),
    # sub-blocks of 27^3 and 32^3: two and one block-wise candidates per
    # launch (their reconstructions side by side in shared memory)
    dict(anchor_stride=8, sub_frac=0.6),
    dict(anchor_stride=8, sub_frac=1.0),
    dict(anchor_stride=8, sub_frac=0.6, allow_natural=0),
])
def test_tune_options(gpu, oracle, kw):
    from paper_2311_12133_gb300 import fields
    x = fields.make("bumps", (50, 44, 39), seed=5)
    xd, g_cfg, o_cfg, _ = _tune_both(gpu, oracle, x, 1e-3, 1, **kw)
    _compress_equal(gpu, oracle, xd, x, 1e-3, 1, g_cfg, o_cfg)


def test_tune_freezes_rough_dim(gpu, oracle):
    """White noise across planes, smooth within them: both sides freeze the
    noisy dim (Sec. 6.3)."""
    rng = np.random.default_rng(3)
    n = 40
    j = np.linspace(0, 2 * np.pi, n)
    plane = np.sin(j)[:, None] * np.cos(j)[None, :]
    x = (plane[None, :, :] * (1 + rng.normal(0, 1, (n, 1, 1)))
         + rng.normal(0, 1, (n, 1, 1))).astype(np.float32)
    xd, g_cfg, o_cfg, o_rep = _tune_both(gpu, oracle, x, 1e-3, 1,
                                         anchor_stride=8, block_rate=0.1)
    assert o_rep.froze == 1 and g_cfg.frozen_dim == 0
    _compress_equal(gpu, oracle, xd, x, 1e-3, 1, g_cfg, o_cfg)


def test_tune_abs_and_1d(gpu, oracle):
    rng = np.random.default_rng(9)
    x1 = np.cumsum(rng.normal(0, 1, 5000)).astype(np.float32)
    xd, g_cfg, o_cfg, _ = _tune_both(gpu, oracle, x1, 0.05, 0)
    _compress_equal(gpu, oracle, xd, x1, 0.05, 0, g_cfg, o_cfg)
    from paper_2311_12133_gb300 import fields
    x3 = fields.make("grf", (33, 34, 35), seed=2)
    xd, g_cfg, o_cfg, _ = _tune_both(gpu, oracle, x3, 0.01, 0)
    _compress_equal(gpu, oracle, xd, x3, 0.01, 0, g_cfg, o_cfg)


def test_tune_integer_lorenzo(gpu, oracle):
    """Integer data at e = 1/2 (exact Lorenzo codes) on small fields."""
    rng = np.random.default_rng(7)
    x = rng.integers(0, 21, size=(33, 33, 33)).astype(np.float32)
    _tune_both(gpu, oracle, x, 0.5, 0, tune_blockwise=0)


def test_tune_constant_and_errors(gpu, oracle):
    import torch
    from paper_2311_12133_gb300 import hpez
    xd = torch.ones((20, 20), dtype=torch.float32, device="cuda")
    cfg, rep = gpu.tune(xd, 1e-3)
    assert cfg.blockwise == 0 and cfg.anchor_stride == 64
    assert rep.stats_count == 0
    x = torch.zeros((20, 20), dtype=torch.float32, device="cuda")
    x[3, 4] = float("nan")
    with pytest.raises(hpez.HpezError) as e:
        gpu.tune(x, 1e-3)
    assert e.value.code == -2
    with pytest.raises(hpez.HpezError) as e:
        gpu.tune(xd, 0.0)
    assert e.value.code == -1
    # sample blocks beyond shared memory: 3D anchor stride 64
    big = torch.rand((70, 70, 70), device="cuda")
    with pytest.raises(hpez.HpezError) as e:
        gpu.tune(big, 1e-3, 1, hpez.hpez_default_tune_params(anchor_stride=64))
    assert e.value.code == -8


def test_tune_full_size_grf512(gpu, oracle):
    """The benchmark field: 512^3 k^-5/3 Gaussian random field, rel eb 1e-3,
    full tuning; theta, block map and report equal the oracle's."""
    import torch
    from paper_2311_12133_gb300 import fields, hpez
    xd = fields.grf_torch((512, 512, 512), seed=0)
    x = xd.cpu().numpy()
    g_cfg, g_rep = gpu.tune(xd, 1e-3)
    o_cfg, o_rep = oracle.tune(x, 1e-3)
    _compare(g_cfg, g_rep, o_cfg, o_rep)
    del xd
    torch.cuda.empty_cache()
