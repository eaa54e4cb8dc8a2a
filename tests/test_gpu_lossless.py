"""Parity of the device lossless stage (Sec. 4, Step 5) with the oracle's:
the encoded bytes are equal, decoding restores the stream exactly, and the
decompressor takes encoded streams directly."""
import struct

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


def _dev(b: bytes):
    import torch
    t = torch.zeros(max(len(b), 16), dtype=torch.uint8, device="cuda")
    t[:len(b)] = torch.frombuffer(bytearray(b), dtype=torch.uint8).cuda()
    return t


def _encode(ctx, s: bytes):
    import torch
    from paper_2311_12133_gb300 import hpez
    d = _dev(s)
    out = torch.empty(len(s) + 64, dtype=torch.uint8, device="cuda")
    n = hpez.hpez_lossless_encode(ctx.handle, d.data_ptr(), len(s), out.data_ptr(), out.numel(),
                                  torch.cuda.current_stream().cuda_stream)
    return out[:n].cpu().numpy().tobytes()


def _decode(ctx, z: bytes, raw: int):
    import torch
    from paper_2311_12133_gb300 import hpez
    d = _dev(z)
    out = torch.empty(raw + 16, dtype=torch.uint8, device="cuda")
    n = hpez.hpez_lossless_decode(ctx.handle, d.data_ptr(), len(z), out.data_ptr(), out.numel(),
                                  torch.cuda.current_stream().cuda_stream)
    return out[:n].cpu().numpy().tobytes()


def _runs(rng, nwords):
    w = []
    while len(w) < nwords:
        v = int(rng.choice([0, 7, 0xFFFFFFFF, int(rng.integers(1, 1 << 31))]))
        w += [v] * int(rng.integers(1, 3000))
    return struct.pack(f"<{nwords}I", *w[:nwords])


@pytest.mark.parametrize("nwords,cut", [(0, 0), (1, 0), (3, 1), (1000, 0), (31, 2),
                                        (1024, 0), (1025, 3), (40000, 1), (2_000_000, 0)])
def test_bodies_equal_oracle(gpu, oracle, nwords, cut):
    """Bodies of runs across blocks and groups, ragged ends, one group to
    many, through a header without flags."""
    rng = np.random.default_rng(nwords + cut)
    body = _runs(rng, nwords)
    body = body[:len(body) - cut] if cut <= len(body) else b""
    s = bytes(512) + body
    want = oracle.lossless_encode(s)
    got = _encode(gpu, s)
    assert got == want
    if got != s:
        assert _decode(gpu, got, len(s)) == s


def test_incompressible_and_refusals(gpu, oracle):
    from paper_2311_12133_gb300 import hpez
    body = np.random.default_rng(0).integers(0, 2 ** 32, 5000, dtype=np.uint64).astype(
        np.uint32).tobytes()
    s = bytes(512) + body
    assert _encode(gpu, s) == s == oracle.lossless_encode(s)
    z = oracle.lossless_encode(bytes(512) + bytes(4 * 9000) + struct.pack("<I", 5) + bytes(40))
    with pytest.raises(hpez.HpezError):  # an encoded stream is not encoded again
        _encode(gpu, z)
    bad = bytearray(z)
    bad[512 + 32] ^= 0x01  # a group-mask bit flipped
    with pytest.raises(hpez.HpezError) as e:
        _decode(gpu, bytes(bad), 512 + 4 * 9011)
    assert e.value.code == -4
    with pytest.raises(hpez.HpezError):
        _decode(gpu, z[:-4], 512 + 4 * 9011)


@pytest.mark.parametrize("kind,shape,eb", [("bumps", (64, 64, 64), 1e-1),
                                           ("bumps", (64, 64, 64), 1e-2),
                                           ("climate2d", (360, 720), 1e-1),
                                           ("grf", (64, 64, 64), 1e-3)])
def test_compressed_streams(gpu, oracle, kind, shape, eb):
    """Compressed fields through the stage: the oracle's bytes, and the
    decompressor on the encoded stream returns the oracle's field."""
    import torch
    from paper_2311_12133_gb300 import fields
    x = fields.make(kind, shape, 4)
    buf, size = gpu.compress(torch.from_numpy(x).cuda(), eb)
    s = buf[:size].cpu().numpy().tobytes()
    want = oracle.lossless_encode(s)
    z = _encode(gpu, s)
    assert z == want and len(z) <= len(s)
    y = gpu.decompress(_dev(z), len(z), shape=shape).cpu().numpy()
    assert y.tobytes() == oracle.decompress(want).tobytes()
