"""Pins of the oracle's lossless stage (Sec. 4, Step 5): run suppression of
repeated 32-bit words of the stream body with two levels of masks.

Checked against a restatement of the format written out here (layout of
worked examples), by exhaustive round trips over every body of up to three
words from a small alphabet, by round trips of real streams through the
oracle's decompressor, and by the rule that a stream it cannot shrink is
returned unchanged.
"""
import itertools
import struct

import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_12133_gb300 import fields

HDR = 512


def _stream(body: bytes) -> bytes:
    """A header of zeros (no flags) followed by `body`."""
    return bytes(HDR) + body


def _words(body: bytes):
    pad = body + bytes((-len(body)) % 4)
    return list(struct.unpack(f"<{len(pad) // 4}I", pad))


def _expected(body: bytes) -> bytes:
    """The format restated: change masks per 32 words, group masks per 32
    blocks, kept masks and words in order."""
    w = _words(body)
    nw = len(w)
    nb = (nw + 31) // 32
    ng = (nb + 31) // 32
    m1 = [0] * nb
    lits = []
    prev = 0
    for i, v in enumerate(w):
        if v != prev:
            m1[i // 32] |= 1 << (i % 32)
            lits.append(v)
        prev = v
    m2 = [0] * ng
    for b, m in enumerate(m1):
        if m:
            m2[b // 32] |= 1 << (b % 32)
    kept = [m for m in m1 if m]
    hdr = bytearray(HDR)
    hdr[8:12] = struct.pack("<I", 2)
    hdr[O.H_RAWSIZE:O.H_RAWSIZE + 8] = struct.pack("<Q", HDR + len(body))
    z = bytes(hdr) + struct.pack("<4Q", nw, len(lits), len(kept), 0)
    z += struct.pack(f"<{ng}I", *m2) + struct.pack(f"<{len(kept)}I", *kept)
    z += struct.pack(f"<{len(lits)}I", *lits)
    return z


def test_worked_layouts():
    # a long run of zeros with one word set: one literal, one mask
    body = bytes(4 * 5000)
    body = body[:4 * 1234] + struct.pack("<I", 7) + body[4 * 1235:]
    z = O.lossless_encode(_stream(body))
    assert z == _expected(body)
    # 157 blocks -> 5 group masks; one block mask; the 7 and the 0 after it
    assert len(z) == HDR + 32 + 4 * (5 + 1 + 2)
    assert O.lossless_decode(z) == _stream(body)
    # all zeros: only the group masks remain
    z = O.lossless_encode(_stream(bytes(4 * 4096)))
    assert len(z) == HDR + 32 + 4 * 4
    # a constant non-zero run: one literal
    body = struct.pack("<I", 0xDEADBEEF) * 3000
    z = O.lossless_encode(_stream(body))
    assert z == _expected(body) and O.lossless_decode(z) == _stream(body)


def test_incompressible_stays_raw():
    body = np.random.default_rng(0).integers(0, 2 ** 32, 1000, dtype=np.uint64).astype(
        np.uint32).tobytes()
    s = _stream(body)
    assert O.lossless_encode(s) == s


def test_exhaustive_small_bodies():
    """Every body of 0-3 words over {0, 1, 0xFFFFFFFF} and every length of a
    ragged last word: encode, decode back (or raw when no gain)."""
    alpha = [0, 1, 0xFFFFFFFF]
    for n in range(0, 4):
        for ws in itertools.product(alpha, repeat=n):
            full = struct.pack(f"<{n}I", *ws)
            for cut in range(max(0, 4 * n - 3), 4 * n + 1):
                body = full[:cut]
                s = _stream(body)
                z = O.lossless_encode(s)
                if z == s:
                    assert len(_expected(body)) >= len(s)
                else:
                    assert z == _expected(body)
                    assert O.lossless_decode(z) == s
    # long runs across block and group boundaries
    rng = np.random.default_rng(3)
    for _ in range(20):
        runs = []
        while sum(len(r) for r in runs) < 3000:
            runs.append([int(rng.choice([0, 5, 0xFFFFFFFF, int(rng.integers(1, 1 << 31))]))]
                        * int(rng.integers(1, 700)))
        w = [v for r in runs for v in r]
        body = struct.pack(f"<{len(w)}I", *w)[:4 * len(w) - int(rng.integers(0, 4))]
        z = O.lossless_encode(_stream(body))
        assert z == _expected(body) and O.lossless_decode(z) == _stream(body)


@pytest.mark.parametrize("eb", [1e-1, 1e-2, 1e-3])
def test_real_streams_round_trip(eb):
    """Compressed fields through the stage and back through the oracle's
    decompressor (which undoes the stage itself)."""
    x = fields.make("bumps", (48, 40, 36), 2)
    s, _, _, recon = O.compress(x, eb, O.EB_REL, want_recon=True)
    z = O.lossless_encode(s)
    assert len(z) <= len(s)
    assert O.decompress(z).tobytes() == recon.tobytes()
    if z != s:
        assert O.lossless_decode(z) == s


def test_corrupt_lossless_streams_rejected():
    body = bytes(4 * 3000) + struct.pack("<I", 9) + bytes(400)
    z = bytearray(O.lossless_encode(_stream(body)))
    bad = bytes(z[:-4])  # a literal missing
    with pytest.raises(O.OracleError):
        O.lossless_decode(bad)
    z2 = bytearray(z)
    z2[HDR + 32] ^= 0x01  # a group-mask bit flipped: the kept masks no longer match
    with pytest.raises(O.OracleError):
        O.lossless_decode(bytes(z2))
