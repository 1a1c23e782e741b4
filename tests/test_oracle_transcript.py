"""Pins of the transcript hash (a test aid with no counterpart in the paper): its mixing function
is the SplitMix64 output function of the published generator, and the hash responds to every
message it covers."""
import numpy as np

import oracle

GAMMA = 0x9E3779B97F4A7C15


def test_mix64_is_splitmix64(golden):
    """SplitMix64 seeded with state 0: state += gamma, output = mix(state)."""
    rows = [r for r in golden("splitmix64_kat.txt")]
    want = [int(r[0], 16) for r in rows]
    got = [oracle.mix64((k + 1) * GAMMA) for k in range(len(want))]
    assert got == want


def _case(rng, n=5, s=37, Q=3, wide=False):
    dt = np.uint32 if wide else np.uint16
    hi = 1 << (32 if wide else 16)
    zc = rng.integers(0, hi, (3, n, s), dtype=np.uint64).astype(dt)
    zm = rng.integers(0, 1 << 32, (3, n, s), dtype=np.uint64).astype(np.uint32)
    bits = rng.integers(0, 2, (3, Q), dtype=np.uint8)
    return zc, zm, bits


def test_transcript_hash_sees_every_message():
    rng = np.random.default_rng(60)
    for wide in (False, True):
        zc, zm, bits = _case(rng, wide=wide)
        h = oracle.transcript_hash(zc, zm, bits)
        assert h == oracle.transcript_hash(zc.copy(), zm.copy(), bits.copy())
        for _ in range(40):
            which = rng.integers(3)
            a, b, c = (x.copy() for x in (zc, zm, bits))
            if which == 0:
                j, n, i = (int(rng.integers(d)) for d in a.shape)
                a[j, n, i] ^= a.dtype.type(1 << int(rng.integers(8 * a.itemsize)))
            elif which == 1:
                j, n, i = (int(rng.integers(d)) for d in b.shape)
                b[j, n, i] ^= np.uint32(1 << int(rng.integers(32)))
            else:
                j, q = (int(rng.integers(d)) for d in c.shape)
                c[j, q] ^= 1
            assert oracle.transcript_hash(a, b, c) != h
        # the same values sent by another party, or for another column, are other messages
        assert oracle.transcript_hash(zc[[1, 0, 2]], zm, bits) != h or (zc[0] == zc[1]).all()
        assert oracle.transcript_hash(zc[:, ::-1].copy(), zm, bits) != h


def test_transcript_hash_is_a_xor_over_messages():
    """Splitting the messages into code, mask and bit parts composes by XOR."""
    rng = np.random.default_rng(61)
    zc, zm, bits = _case(rng)
    zero_bits = np.zeros_like(bits)
    h_all = oracle.transcript_hash(zc, zm, bits)
    h_code_bits = oracle.transcript_hash(zc, None, bits)
    h_code = oracle.transcript_hash(zc, None, zero_bits)
    h_code_mask = oracle.transcript_hash(zc, zm, zero_bits)
    assert h_all ^ h_code_bits == h_code_mask ^ h_code
