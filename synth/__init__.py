"""Seeded synthetic workloads for the iris uniqueness check.

This module holds none of the method's arithmetic: it only turns
(seed, stream, index) into iris-code bits, mask bits and the choices that plant
near-duplicate queries. Both the CPU oracle and the GPU path take their inputs
from here. The host implementation is numpy; ``synth_gen.cu`` implements the
same database-bit generator on the device for databases too large to build on
the host, and a GPU test checks the two agree.

Generator: the SplitMix64 output function (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style:
    mix(z)      = z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27;
                  z *= 0x94D049BB133111EB; z ^= z>>31
    h(s, t, i)  = mix( mix(s ^ (t << 56)) + (i + 1) * 0x9E3779B97F4A7C15 )
Bits are packed 64 per uint64 word, bit b of a row in word b//64 at b%64.
Code bits are Bernoulli(1/2) (the raw hash bits). A mask bit is set when its
16-bit draw is below 58982 (p = 0.89999, the workloads' Bernoulli(0.9)).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
MASK_P16 = 58982

S_DB_CODE, S_DB_MASK, S_Q_CODE, S_Q_MASK, S_PLANT, S_FLIP, S_PICK = 1, 2, 3, 4, 5, 6, 7


def mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z ^ (z >> np.uint64(30))
        z = z * M1
        z = z ^ (z >> np.uint64(27))
        z = z * M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_base(seed: int, stream: int) -> np.uint64:
    return mix64(np.uint64((int(seed) ^ (int(stream) << 56)) & 0xFFFFFFFFFFFFFFFF))


def h(seed: int, stream: int, idx) -> np.ndarray:
    """Counter-style hash h(seed, stream, idx) for an array of indices."""
    base = stream_base(seed, stream)
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(base + (idx + np.uint64(1)) * GAMMA)


def _row_bits(seed: int, s_code: int, s_mask: int, rows, l: int):
    rows = np.asarray(rows, dtype=np.uint64)
    nw = (l + 63) // 64
    nd = (l + 3) // 4
    code = h(seed, s_code, rows[:, None] * np.uint64(nw) + np.arange(nw, dtype=np.uint64)[None, :])
    draws = h(seed, s_mask, rows[:, None] * np.uint64(nd) + np.arange(nd, dtype=np.uint64)[None, :])
    # 4 sixteen-bit draws per hash: bit 4t+j uses bits 16j..16j+15 of draw t
    d16 = ((draws[:, :, None] >> (np.uint64(16) * np.arange(4, dtype=np.uint64))[None, None, :])
           & np.uint64(0xFFFF)).reshape(len(rows), nd * 4)[:, :l]
    mbits = (d16 < MASK_P16)
    mask = pack_bits(mbits)
    code = code.copy()
    if l % 64:
        keep = np.uint64((1 << (l % 64)) - 1)
        code[:, -1] &= keep
    return code, mask


def db_bits(seed: int, rows, l: int = 12800):
    """Code and mask bits of the database rows with the given indices: ([n][nw], [n][nw]) uint64."""
    return _row_bits(seed, S_DB_CODE, S_DB_MASK, rows, l)


def random_query_bits(seed: int, qidx, l: int = 12800):
    return _row_bits(seed, S_Q_CODE, S_Q_MASK, qidx, l)


def pack_bits(bits) -> np.ndarray:
    """[n][l] bool -> [n][ceil(l/64)] uint64, bit b in word b//64 at position b%64."""
    bits = np.asarray(bits, dtype=bool)
    n, l = bits.shape
    nw = (l + 63) // 64
    pad = np.zeros((n, nw * 64), dtype=bool)
    pad[:, :l] = bits
    by = np.packbits(pad, axis=-1, bitorder="little")
    return np.ascontiguousarray(by).view("<u8").reshape(n, nw).astype(np.uint64)


def unpack_bits(words, l: int) -> np.ndarray:
    words = np.ascontiguousarray(np.asarray(words, dtype=np.uint64))
    n, nw = words.shape
    by = words.view(np.uint8).reshape(n, nw, 8)
    bits = np.unpackbits(by, axis=-1, bitorder="little").reshape(n, nw * 64)
    return bits[:, :l].astype(bool)


def shift_columns(bits, rows: int, cols: int, cell: int, u: int) -> np.ndarray:
    """Cyclic column shift of unpacked codes: out[r][j][k] = in[r][(j-u) mod cols][k]."""
    b = np.asarray(bits).reshape(-1, rows, cols, cell)
    return np.roll(b, u, axis=2).reshape(len(b), rows * cols * cell)


@dataclass
class Workload:
    """A seeded workload: database size, queries, rotations and planted near-duplicates."""
    name: str
    s: int
    Q: int
    rot_lo: int = -15
    R: int = 31
    planted: int = 0
    flip: float | tuple = 0.10
    seed: int = 0x1A150001
    rows: int = 16
    cols: int = 200
    cell: int = 4
    db_share_seed: int = 0xDB5EED
    q_share_seed: int = 0x0E5EED
    prf_seeds: tuple = (0x51EED0, 0x51EED1, 0x51EED2)
    thr_a: int = 16384
    extra: dict = field(default_factory=dict)

    @property
    def l(self) -> int:
        return self.rows * self.cols * self.cell

    @property
    def nwords(self) -> int:
        return (self.l + 63) // 64

    @property
    def comparisons(self) -> int:
        return self.s * self.Q * self.R

    def planted_set(self) -> np.ndarray:
        """Indices of the planted queries: the first `planted` entries of a seeded permutation."""
        perm = np.arange(self.Q)
        if self.planted <= 0:
            return perm[:0]
        r = h(self.seed, S_PICK, np.arange(self.Q))
        for t in range(self.Q - 1):
            j = t + int(r[t] % np.uint64(self.Q - t))
            perm[t], perm[j] = perm[j], perm[t]
        return np.sort(perm[: self.planted])

    def plant(self, q: int) -> dict:
        """Source row, column offset and flipped positions of planted query q."""
        d = h(self.seed, S_PLANT, np.arange(3 * q, 3 * q + 3))
        src = int(d[0] % np.uint64(self.s))
        u = 0 if (int(d[1]) & 1) == 0 else int((int(d[1]) >> 1) % 31) - 15
        if isinstance(self.flip, tuple):
            frac = (int(d[2]) >> 11) / float(1 << 53)
            rate = self.flip[0] + (self.flip[1] - self.flip[0]) * frac
        else:
            rate = float(self.flip)
        F = int(np.floor(rate * self.l + 0.5))
        l = self.l
        perm = np.arange(l)
        r = h(self.seed, S_FLIP, np.uint64(q) * np.uint64(l) + np.arange(F, dtype=np.uint64))
        for t in range(F):
            j = t + int(r[t] % np.uint64(l - t))
            perm[t], perm[j] = perm[j], perm[t]
        return {"src": src, "u": u, "flips": np.sort(perm[:F]), "rate": rate}

    def db_bits(self, rows=None):
        if rows is None:
            rows = np.arange(self.s)
        return db_bits(self.seed, rows, self.l)

    def query_bits(self):
        """Packed code/mask bits of all queries, with planted near-duplicates in place."""
        qc, qm = random_query_bits(self.seed, np.arange(self.Q), self.l)
        for q in self.planted_set():
            p = self.plant(int(q))
            c, m = db_bits(self.seed, [p["src"]], self.l)
            cb = unpack_bits(c, self.l)
            mb = unpack_bits(m, self.l)
            cb = shift_columns(cb, self.rows, self.cols, self.cell, p["u"])
            mb = shift_columns(mb, self.rows, self.cols, self.cell, p["u"])
            cb[0, p["flips"]] ^= True
            qc[q] = pack_bits(cb)[0]
            qm[q] = pack_bits(mb)[0]
        return qc, qm


def workload(name: str) -> Workload:
    """The named workloads: tiny, plain-vs-precision, planted, serving, largest."""
    if name in ("c1", "tiny"):
        return Workload("tiny: 1000 x 4 queries, no rotations", s=1000, Q=4, rot_lo=0, R=1, planted=0,
                        seed=0x1A150001)
    if name in ("c2", "plain_vs_precision"):
        return Workload("plain-vs-precision: 100000 x 32 queries x 31 rotations", s=100_000, Q=32, planted=4,
                        seed=0x1A150002)
    if name in ("c3", "planted"):
        return Workload("planted: 500000 x 64 queries x 31 rotations", s=500_000, Q=64, planted=32,
                        seed=0x1A150003)
    if name in ("c4", "serving"):
        return Workload("serving: 250000 rows, batches of 1..256 queries x 31 rotations", s=250_000, Q=256,
                        planted=13, seed=0x1A150004)
    if name in ("c5", "largest"):
        return Workload("largest: 600000 x 256 queries x 31 rotations", s=600_000, Q=256, planted=13,
                        flip=(0.05, 0.15), seed=0x1A150005)
    raise KeyError(name)


# ----------------------------------------------------------------------------------------
# Device half (synth_gen.cu -> libsynth.so): the same database-bit generator on the GPU.
# ----------------------------------------------------------------------------------------
_synth_lib = None


def _device_lib():
    global _synth_lib
    if _synth_lib is None:
        import ctypes
        import os
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsynth.so")
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: run the package build first")
        L = ctypes.CDLL(path)
        L.synth_db_bits.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.synth_db_bits.restype = ctypes.c_int
        _synth_lib = L
    return _synth_lib


def device_db_bits(seed: int, row0: int, n: int, l: int, code_ptr: int, mask_ptr: int, stream: int | None = None):
    """Write the packed code/mask bits of rows row0..row0+n-1 to device buffers [n][ceil(l/64)] uint64."""
    rc = _device_lib().synth_db_bits(seed & 0xFFFFFFFFFFFFFFFF, row0, n, l, code_ptr, mask_ptr, stream)
    if rc != 0:
        raise RuntimeError("synth_db_bits launch failed")
