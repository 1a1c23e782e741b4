"""CPU oracle for the share-domain iris uniqueness check -- TEST INFRASTRUCTURE ONLY.

A plain, slow restatement of arXiv 2405.04463 (Alg. 1, Alg. 3, App. C, App. D)
in C (``oracle.c``), wrapped here with ctypes and numpy. Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package; the CUDA library shares no code with it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

D_SHARE, D_ZA, D_AND, D_INJ0, D_INJ2, D_OR = 1, 2, 3, 4, 5, 6
D_SHARE32, D_ZA32 = 9, 10
LIFT_CONST, LIFT_NONE = 1, 2   # lifting variants (Sec. 5.1, Sec. 6.2)
LIFT_GATE0, MSB_GATE0 = 0, 36


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (OpenMP when available)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if not (force or stale):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", _SRC, "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


class Geom(ctypes.Structure):
    """Code geometry rows x cols x cell (bit (r*cols+j)*cell+k) and rotations rot_lo..rot_lo+R-1."""
    _fields_ = [("rows", ctypes.c_uint32), ("cols", ctypes.c_uint32), ("cell", ctypes.c_uint32),
                ("rot_lo", ctypes.c_int32), ("R", ctypes.c_uint32)]

    @property
    def l(self) -> int:
        return self.rows * self.cols * self.cell

    @property
    def nwords(self) -> int:
        return (self.l + 63) // 64


def iris_geom(rot_lo: int = -15, R: int = 31) -> Geom:
    """The deployed geometry: 16 x 200 x 4 = 12800 bits (Sec. 3)."""
    return Geom(16, 200, 4, rot_lo, R)


class MpcCfg(ctypes.Structure):
    _fields_ = [("seeds", ctypes.c_uint64 * 3), ("req", ctypes.c_uint32), ("thr_a", ctypes.c_uint32)]


def mpc_cfg(seeds=(0x5EED0, 0x5EED1, 0x5EED2), req: int = 0, thr_a: int = 16384) -> MpcCfg:
    c = MpcCfg()
    for j in range(3):
        c.seeds[j] = int(seeds[j]) & 0xFFFFFFFFFFFFFFFF
    c.req = req
    c.thr_a = thr_a
    return c


class Stats(ctypes.Structure):
    _fields_ = [("and_gates", ctypes.c_uint64), ("bits_sent", ctypes.c_uint64 * 3),
                ("depth_lift", ctypes.c_uint32), ("depth_msb", ctypes.c_uint32),
                ("depth_total", ctypes.c_uint32), ("depth_or", ctypes.c_uint32),
                ("and_lift", ctypes.c_uint32), ("and_msb", ctypes.c_uint32),
                ("replication_errors", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {"and_gates": self.and_gates, "bits_sent": list(self.bits_sent),
                "depth_lift": self.depth_lift, "depth_msb": self.depth_msb,
                "depth_total": self.depth_total, "depth_or": self.depth_or,
                "and_lift": self.and_lift, "and_msb": self.and_msb,
                "replication_errors": self.replication_errors}


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


def _p(t):
    return ctypes.POINTER(t)


def _declare(L):
    u8, u16, u32, u64, i32 = ctypes.c_uint8, ctypes.c_uint16, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32
    G, C, S = _p(Geom), _p(MpcCfg), _p(Stats)
    L.orc_philox4x32_10.argtypes = [_p(u32), _p(u32), _p(u32)]
    L.orc_rotate_u16.argtypes = [G, _p(u16), _p(u16), i32]
    L.orc_rotate_bits.argtypes = [G, _p(u64), _p(u64), i32]
    L.orc_encode_share.argtypes = [_p(u64), _p(u64), u32, u32, u64, u32, u32, _p(u16), _p(u16)]
    L.orc_plain_pair.argtypes = [_p(u64), _p(u64), _p(u64), _p(u64), u32, _p(i32), _p(i32)]
    L.orc_plain_match.argtypes = [G, _p(u64), _p(u64), u32, _p(u64), _p(u64), u32, ctypes.c_int,
                                  u32, u32, u32, _p(i32), _p(i32), _p(u8), ctypes.c_int]
    L.orc_mpc_dot.argtypes = [C, _p(u16), u64, _p(u16), u64, u32, u32, u32, u32, u32, _p(u16), S]
    L.orc_mpc_compare.argtypes = [C, _p(u16), _p(u16), u32, u32, u32, _p(u8), _p(u32), _p(u32), S]
    L.orc_bit_extract.argtypes = [C, _p(u32), u32, u32, u32, u32, u32, _p(u8), _p(u8), S]
    L.orc_or_tree.argtypes = [C, _p(u8), u32, u32, u32, _p(u8), S]
    L.orc_bit_extract_batch.argtypes = [C, _p(u32), u32, u32, u32, _p(u8), _p(u8)]
    L.orc_gr_mul.argtypes = [_p(u16), _p(u16), _p(u16)]
    L.orc_gr_inv.argtypes = [_p(u16), _p(u16)]
    L.orc_gr_inv.restype = ctypes.c_int
    L.orc_gr_points.argtypes = [_p(u16)]
    L.orc_gr_lagrange.argtypes = [_p(u16)]
    L.orc_encode_share_galois.argtypes = [_p(u64), _p(u64), u32, u32, u64, u32, u32, _p(u16), _p(u16)]
    L.orc_mpc_dot_galois.argtypes = [C, _p(u16), u64, _p(u16), u64, u32, u32, u32, u32, u32, _p(u16), S]
    L.orc_mpc_match_galois.argtypes = [C, G, _p(u16), _p(u16), u32, _p(u16), _p(u16), u32,
                                       _p(u16), _p(u16), _p(u8), _p(u8), S]
    L.orc_mpc_compare_plain.argtypes = [C, _p(u16), u32, u32, u32, u32, _p(u8), S]
    L.orc_mpc_match_plain.argtypes = [C, G, ctypes.c_int, _p(u16), _p(u64), u32, _p(u16), _p(u64), u32,
                                      _p(u16), _p(u16), _p(u8), S]
    L.orc_mpc_match_batch.argtypes = [C, G, ctypes.c_int, _p(u16), _p(u16), u32, _p(u8), S]
    L.orc_or_combine.argtypes = [C, _p(u8), u32, _p(u8), S]
    L.orc_mpc_match.argtypes = [C, G, _p(u16), _p(u16), u32, _p(u16), _p(u16), u32,
                                _p(u16), _p(u16), _p(u8), _p(u8), S]
    vp = ctypes.c_void_p
    L.orc_mix64.argtypes = [u64]
    L.orc_mix64.restype = u64
    L.orc_transcript_hash.argtypes = [vp, u32, vp, u32, u32, u32, _p(u8), u32]
    L.orc_transcript_hash.restype = u64
    L.orc_encode_share32.argtypes = [_p(u64), _p(u64), u32, u32, u64, u32, u32, _p(u32), _p(u32)]
    L.orc_mpc_dot32.argtypes = [C, _p(u32), u64, _p(u32), u64, u32, u32, u32, u32, u32, _p(u32), S]
    L.orc_mpc_compare_liftfree.argtypes = [C, ctypes.c_int, _p(u32), _p(u32), u32, u32, u32, u32, _p(u8), _p(u32), S]
    L.orc_mpc_match_lift.argtypes = [C, G, ctypes.c_int, u32, vp, _p(u32), u32, vp, _p(u32), u32, vp, _p(u32),
                                     _p(u8), S]
    for f in ("orc_philox4x32_10", "orc_rotate_u16", "orc_rotate_bits", "orc_encode_share", "orc_plain_pair",
              "orc_plain_match", "orc_mpc_dot", "orc_mpc_compare", "orc_bit_extract", "orc_or_tree",
              "orc_mpc_match"):
        getattr(L, f).restype = None


def _ptr(a, t):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(t))


# ----------------------------------------------------------------------------------------
# Wrappers
# ----------------------------------------------------------------------------------------

def philox(key, ctr) -> np.ndarray:
    """Philox4x32-10 (Salmon et al., SC'11) of a 4-word counter under a 2-word key."""
    k = np.ascontiguousarray(key, dtype=np.uint32)
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(k, ctypes.c_uint32), _ptr(c, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def rotate_u16(g: Geom, v, shift: int) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.uint16)
    out = np.empty_like(v)
    lib().orc_rotate_u16(ctypes.byref(g), _ptr(v, ctypes.c_uint16), _ptr(out, ctypes.c_uint16), shift)
    return out


def rotate_bits(g: Geom, v, shift: int) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.uint64)
    out = np.empty_like(v)
    lib().orc_rotate_bits(ctypes.byref(g), _ptr(v, ctypes.c_uint64), _ptr(out, ctypes.c_uint64), shift)
    return out


def encode_share(code_bits, mask_bits, l: int, client_seed: int, side: int, idx0: int = 0):
    """Masked-bit encoding and client sharing of packed rows; returns code, mask shares [3][n][l] u16."""
    cb = np.ascontiguousarray(code_bits, dtype=np.uint64)
    mb = np.ascontiguousarray(mask_bits, dtype=np.uint64)
    n = cb.shape[0]
    code = np.empty((3, n, l), np.uint16)
    mask = np.empty((3, n, l), np.uint16)
    lib().orc_encode_share(_ptr(cb, ctypes.c_uint64), _ptr(mb, ctypes.c_uint64), n, l,
                           client_seed & 0xFFFFFFFFFFFFFFFF, side, idx0,
                           _ptr(code, ctypes.c_uint16), _ptr(mask, ctypes.c_uint16))
    return code, mask


def plain_pair(c, m, C, M):
    c, m, C, M = (np.ascontiguousarray(a, dtype=np.uint64) for a in (c, m, C, M))
    ml, hd = ctypes.c_int32(), ctypes.c_int32()
    lib().orc_plain_pair(_ptr(c, ctypes.c_uint64), _ptr(m, ctypes.c_uint64), _ptr(C, ctypes.c_uint64),
                         _ptr(M, ctypes.c_uint64), c.shape[-1], ctypes.byref(ml), ctypes.byref(hd))
    return ml.value, hd.value


def plain_match(g: Geom, qc, qm, dc, dm, rule: int = 0, tau=(3, 8), thr_a: int = 16384,
                distances: bool = False, threads: int = 1):
    """Alg. 1 with rotations. Returns (match[Q], ml[Q][R][s] | None, hd[Q][R][s] | None)."""
    qc, qm, dc, dm = (np.ascontiguousarray(a, dtype=np.uint64) for a in (qc, qm, dc, dm))
    Q, s = qc.shape[0], dc.shape[0]
    match = np.zeros(Q, np.uint8)
    ml = hd = None
    if distances:
        ml = np.zeros((Q, g.R, s), np.int32)
        hd = np.zeros((Q, g.R, s), np.int32)
    lib().orc_plain_match(ctypes.byref(g), _ptr(qc, ctypes.c_uint64), _ptr(qm, ctypes.c_uint64), Q,
                          _ptr(dc, ctypes.c_uint64), _ptr(dm, ctypes.c_uint64), s, rule, tau[0], tau[1],
                          thr_a, _ptr(ml, ctypes.c_int32), _ptr(hd, ctypes.c_int32),
                          _ptr(match, ctypes.c_uint8), threads)
    return match, ml, hd


def mpc_dot(cfg: MpcCfg, x, y, q: int, rho: int, i: int, vec: int, stats: Stats | None = None):
    """App. C dot of DB share row x[3][l] with rotated query shares y[3][l] -> z[3] u16."""
    x = np.ascontiguousarray(x, dtype=np.uint16)
    y = np.ascontiguousarray(y, dtype=np.uint16)
    l = x.shape[-1]
    z = np.zeros(3, np.uint16)
    st = stats if stats is not None else Stats()
    lib().orc_mpc_dot(ctypes.byref(cfg), _ptr(x, ctypes.c_uint16), l, _ptr(y, ctypes.c_uint16), l, l,
                      q, rho, i, vec, _ptr(z, ctypes.c_uint16), ctypes.byref(st))
    return z


def mpc_compare(cfg: MpcCfg, dot, ml, q: int, rho: int, i: int, stats: Stats | None = None):
    """Lift + threshold + MSB of one comparison. Returns (msb[3], ml_lift[3], v[3])."""
    d = np.ascontiguousarray(dot, dtype=np.uint16)
    m = np.ascontiguousarray(ml, dtype=np.uint16)
    msb = np.zeros(3, np.uint8)
    mll = np.zeros(3, np.uint32)
    v = np.zeros(3, np.uint32)
    st = stats if stats is not None else Stats()
    lib().orc_mpc_compare(ctypes.byref(cfg), _ptr(d, ctypes.c_uint16), _ptr(m, ctypes.c_uint16), q, rho, i,
                          _ptr(msb, ctypes.c_uint8), _ptr(mll, ctypes.c_uint32), _ptr(v, ctypes.c_uint32),
                          ctypes.byref(st))
    return msb, mll, v


def bit_extract(cfg: MpcCfg, x, m: int, q: int = 0, rho: int = 0, i: int = 0, gate0: int = MSB_GATE0,
                stats: Stats | None = None):
    """BitExtract of bits m and m-1 of x_0+x_1+x_2 mod 2^32. Returns (top[3], below[3])."""
    xx = np.ascontiguousarray(np.asarray(x, dtype=np.uint64) & 0xFFFFFFFF, dtype=np.uint32)
    top = np.zeros(3, np.uint8)
    below = np.zeros(3, np.uint8)
    st = stats if stats is not None else Stats()
    lib().orc_bit_extract(ctypes.byref(cfg), _ptr(xx, ctypes.c_uint32), m, q, rho, i, gate0,
                          _ptr(top, ctypes.c_uint8), _ptr(below, ctypes.c_uint8), ctypes.byref(st))
    return top, below


def bit_extract_batch(cfg: MpcCfg, x, m: int, gate0: int = 0):
    """orc_bit_extract over rows of x [n][3] (row i at counter row i) -> (top [n][3], below [n][3])."""
    x = np.ascontiguousarray(x, dtype=np.uint32)
    n = x.shape[0]
    top = np.zeros((n, 3), np.uint8)
    below = np.zeros((n, 3), np.uint8)
    lib().orc_bit_extract_batch(ctypes.byref(cfg), _ptr(x, ctypes.c_uint32), n, m, gate0,
                                _ptr(top, ctypes.c_uint8), _ptr(below, ctypes.c_uint8))
    return top, below


def or_tree(cfg: MpcCfg, msb, q: int = 0, stats: Stats | None = None):
    """OR tree of one query over msb[3][R][s] bit components -> bit[3]."""
    msb = np.ascontiguousarray(msb, dtype=np.uint8)
    _, R, s = msb.shape
    bit = np.zeros(3, np.uint8)
    st = stats if stats is not None else Stats()
    lib().orc_or_tree(ctypes.byref(cfg), _ptr(msb, ctypes.c_uint8), R, s, q, _ptr(bit, ctypes.c_uint8),
                      ctypes.byref(st))
    return bit


def mpc_match(cfg: MpcCfg, g: Geom, db_code, db_mask, q_code, q_mask, want_z: bool = False,
              want_msb: bool = False):
    """Alg. 3 for all queries. Shares are [3][n][l] u16. Returns a dict with bits[3][Q]
    (and z_code/z_mask [3][Q*R][s], msb [3][Q*R][s] when asked) plus stats."""
    return _mpc_match(lib().orc_mpc_match, cfg, g, db_code, db_mask, q_code, q_mask, want_z, want_msb)


def _mpc_match(fn, cfg, g, db_code, db_mask, q_code, q_mask, want_z, want_msb):
    db_code = np.ascontiguousarray(db_code, dtype=np.uint16)
    db_mask = np.ascontiguousarray(db_mask, dtype=np.uint16)
    q_code = np.ascontiguousarray(q_code, dtype=np.uint16)
    q_mask = np.ascontiguousarray(q_mask, dtype=np.uint16)
    s, Q = db_code.shape[1], q_code.shape[1]
    assert db_code.shape[2] == g.l and q_code.shape[2] == g.l
    n = Q * g.R
    zc = np.zeros((3, n, s), np.uint16) if want_z else None
    zm = np.zeros((3, n, s), np.uint16) if want_z else None
    msb = np.zeros((3, n, s), np.uint8) if want_msb else None
    bits = np.zeros((3, Q), np.uint8)
    st = Stats()
    fn(ctypes.byref(cfg), ctypes.byref(g), _ptr(db_code, ctypes.c_uint16), _ptr(db_mask, ctypes.c_uint16), s,
       _ptr(q_code, ctypes.c_uint16), _ptr(q_mask, ctypes.c_uint16), Q, _ptr(zc, ctypes.c_uint16),
       _ptr(zm, ctypes.c_uint16), _ptr(msb, ctypes.c_uint8), _ptr(bits, ctypes.c_uint8), ctypes.byref(st))
    return {"bits": bits, "z_code": zc, "z_mask": zm, "msb": msb, "stats": st.as_dict()}


# ---- Galois-ring Shamir dot products (Sec. 4.3.2): GR = Z_{2^16}[X]/(X^2 - X - 1) ----

def gr_mul(a, b) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint16)
    b = np.ascontiguousarray(b, dtype=np.uint16)
    out = np.zeros(2, np.uint16)
    lib().orc_gr_mul(_ptr(a, ctypes.c_uint16), _ptr(b, ctypes.c_uint16), _ptr(out, ctypes.c_uint16))
    return out


def gr_inv(a):
    """a^-1, or None if a is not a unit of GR."""
    a = np.ascontiguousarray(a, dtype=np.uint16)
    out = np.zeros(2, np.uint16)
    ok = lib().orc_gr_inv(_ptr(a, ctypes.c_uint16), _ptr(out, ctypes.c_uint16))
    return out if ok else None


def gr_points() -> np.ndarray:
    out = np.zeros(6, np.uint16)
    lib().orc_gr_points(_ptr(out, ctypes.c_uint16))
    return out.reshape(3, 2)


def gr_lagrange() -> np.ndarray:
    out = np.zeros(6, np.uint16)
    lib().orc_gr_lagrange(_ptr(out, ctypes.c_uint16))
    return out.reshape(3, 2)


def encode_share_galois(code_bits, mask_bits, l: int, client_seed: int, side: int, idx0: int = 0):
    """Masked-bit encoding and Galois-ring Shamir sharing (degree 1) of packed rows; returns the
    three parties' code and mask shares [3][n][l] u16 (element e's coefficients at 2e, 2e+1)."""
    cb = np.ascontiguousarray(code_bits, dtype=np.uint64)
    mb = np.ascontiguousarray(mask_bits, dtype=np.uint64)
    n = cb.shape[0]
    code = np.empty((3, n, l), np.uint16)
    mask = np.empty((3, n, l), np.uint16)
    lib().orc_encode_share_galois(_ptr(cb, ctypes.c_uint64), _ptr(mb, ctypes.c_uint64), n, l,
                                  client_seed & 0xFFFFFFFFFFFFFFFF, side, idx0,
                                  _ptr(code, ctypes.c_uint16), _ptr(mask, ctypes.c_uint16))
    return code, mask


def mpc_dot_galois(cfg: MpcCfg, x, y, q: int, rho: int, i: int, vec: int, stats: Stats | None = None):
    """Galois-ring Shamir dot of DB shares x[3][l] with rotated query shares y[3][l] -> z[3]."""
    x = np.ascontiguousarray(x, dtype=np.uint16)
    y = np.ascontiguousarray(y, dtype=np.uint16)
    l = x.shape[-1]
    z = np.zeros(3, np.uint16)
    st = stats if stats is not None else Stats()
    lib().orc_mpc_dot_galois(ctypes.byref(cfg), _ptr(x, ctypes.c_uint16), l, _ptr(y, ctypes.c_uint16), l, l,
                             q, rho, i, vec, _ptr(z, ctypes.c_uint16), ctypes.byref(st))
    return z


def mpc_match_galois(cfg: MpcCfg, g: Geom, db_code, db_mask, q_code, q_mask, want_z: bool = False,
                     want_msb: bool = False):
    """mpc_match with the dot products on Galois-ring Shamir shares (encode_share_galois)."""
    return _mpc_match(lib().orc_mpc_match_galois, cfg, g, db_code, db_mask, q_code, q_mask, want_z, want_msb)


# ---- protocol 1 (Sec. 4, Alg. 2): shared codes, public masks ----

def mpc_compare_plain(cfg: MpcCfg, dot, ml: int, q: int = 0, rho: int = 0, i: int = 0,
                      stats: Stats | None = None):
    """MSB(floor(a ml / 2^16) - dot) on the dot components dot[3] with public ml -> msb[3]."""
    d = np.ascontiguousarray(dot, dtype=np.uint16)
    out = np.zeros(3, np.uint8)
    st = stats if stats is not None else Stats()
    lib().orc_mpc_compare_plain(ctypes.byref(cfg), _ptr(d, ctypes.c_uint16), ml, q, rho, i,
                                _ptr(out, ctypes.c_uint8), ctypes.byref(st))
    return out


def mpc_match_plain(cfg: MpcCfg, g: Geom, db_code, db_mask_bits, q_code, q_mask_bits, galois: bool = False,
                    want_z: bool = False):
    """Alg. 2: code shares [3][n][l] (additive or Galois), plain mask bits [n][words]."""
    db_code = np.ascontiguousarray(db_code, dtype=np.uint16)
    q_code = np.ascontiguousarray(q_code, dtype=np.uint16)
    dm = np.ascontiguousarray(db_mask_bits, dtype=np.uint64)
    qm = np.ascontiguousarray(q_mask_bits, dtype=np.uint64)
    s, Q = db_code.shape[1], q_code.shape[1]
    n = Q * g.R
    zc = np.zeros((3, n, s), np.uint16) if want_z else None
    ml = np.zeros((n, s), np.uint16) if want_z else None
    bits = np.zeros((3, Q), np.uint8)
    st = Stats()
    lib().orc_mpc_match_plain(ctypes.byref(cfg), ctypes.byref(g), int(galois), _ptr(db_code, ctypes.c_uint16),
                              _ptr(dm, ctypes.c_uint64), s, _ptr(q_code, ctypes.c_uint16), _ptr(qm, ctypes.c_uint64),
                              Q, _ptr(zc, ctypes.c_uint16), _ptr(ml, ctypes.c_uint16), _ptr(bits, ctypes.c_uint8),
                              ctypes.byref(st))
    return {"bits": bits, "z_code": zc, "ml": ml, "stats": st.as_dict()}


# ---- both eyes and inner-batch matching (Sec. 5.4) ----

def mpc_match_batch(cfg: MpcCfg, g: Geom, q_code, q_mask, galois: bool = False):
    """Inner-batch part of one eye: query q against the unrotated codes of persons p' < q of the
    same batch (shares [3][P][l]); returns bits [3][P]."""
    q_code = np.ascontiguousarray(q_code, dtype=np.uint16)
    q_mask = np.ascontiguousarray(q_mask, dtype=np.uint16)
    P = q_code.shape[1]
    bits = np.zeros((3, P), np.uint8)
    st = Stats()
    lib().orc_mpc_match_batch(ctypes.byref(cfg), ctypes.byref(g), int(galois), _ptr(q_code, ctypes.c_uint16),
                              _ptr(q_mask, ctypes.c_uint16), P, _ptr(bits, ctypes.c_uint8), ctypes.byref(st))
    return bits


def or_combine(cfg: MpcCfg, bits4) -> np.ndarray:
    """(b0 OR b1) OR (b2 OR b3) per person on boolean sharings bits4 [4][3][P] -> [3][P]."""
    bits4 = np.ascontiguousarray(bits4, dtype=np.uint8)
    P = bits4.shape[2]
    out = np.zeros((3, P), np.uint8)
    st = Stats()
    lib().orc_or_combine(ctypes.byref(cfg), _ptr(bits4, ctypes.c_uint8), P, _ptr(out, ctypes.c_uint8),
                         ctypes.byref(st))
    return out


def reconstruct_u16(shares) -> np.ndarray:
    """Sum of the three additive components mod 2^16 (axis 0)."""
    s = np.asarray(shares).astype(np.uint32)
    return ((s[0] + s[1] + s[2]) & 0xFFFF).astype(np.uint16)


def reconstruct_bits(shares) -> np.ndarray:
    s = np.asarray(shares).astype(np.uint8)
    return (s[0] ^ s[1] ^ s[2]) & 1


# ---- lifting variants (Sec. 5.1, Sec. 6.2 Table 2): ConstLift and NoLift ----

def encode_share32(code_bits, mask_bits, l: int, client_seed: int, side: int, idx0: int = 0):
    """Masked-bit encoding and client sharing over Z_{2^32}: code, mask shares [3][n][l] u32."""
    cb = np.ascontiguousarray(code_bits, dtype=np.uint64)
    mb = np.ascontiguousarray(mask_bits, dtype=np.uint64)
    n = cb.shape[0]
    code = np.empty((3, n, l), np.uint32)
    mask = np.empty((3, n, l), np.uint32)
    lib().orc_encode_share32(_ptr(cb, ctypes.c_uint64), _ptr(mb, ctypes.c_uint64), n, l,
                             client_seed & 0xFFFFFFFFFFFFFFFF, side, idx0,
                             _ptr(code, ctypes.c_uint32), _ptr(mask, ctypes.c_uint32))
    return code, mask


def mpc_dot32(cfg: MpcCfg, x, y, q: int, rho: int, i: int, vec: int, stats: Stats | None = None):
    """App. C dot over Z_{2^32} of DB share row x[3][l] with rotated query shares y[3][l] -> z[3]."""
    x = np.ascontiguousarray(x, dtype=np.uint32)
    y = np.ascontiguousarray(y, dtype=np.uint32)
    l = x.shape[-1]
    z = np.zeros(3, np.uint32)
    st = stats if stats is not None else Stats()
    lib().orc_mpc_dot32(ctypes.byref(cfg), _ptr(x, ctypes.c_uint32), l, _ptr(y, ctypes.c_uint32), l, l,
                        q, rho, i, vec, _ptr(z, ctypes.c_uint32), ctypes.byref(st))
    return z


def mpc_compare_liftfree(cfg: MpcCfg, mode: int, dot, ml, thr_b: int = 0, q: int = 0, rho: int = 0, i: int = 0,
                         stats: Stats | None = None):
    """MSB(a ml - b dot) over Z_{2^32} without Lift: ml components over Z_{2^32}, dot components
    over Z_{2^16} (LIFT_CONST) or Z_{2^32} (LIFT_NONE, b = thr_b). Returns (msb[3], v[3])."""
    d = np.ascontiguousarray(np.asarray(dot, dtype=np.uint64).astype(np.uint32))
    m = np.ascontiguousarray(np.asarray(ml, dtype=np.uint64).astype(np.uint32))
    msb = np.zeros(3, np.uint8)
    v = np.zeros(3, np.uint32)
    st = stats if stats is not None else Stats()
    lib().orc_mpc_compare_liftfree(ctypes.byref(cfg), mode, _ptr(d, ctypes.c_uint32), _ptr(m, ctypes.c_uint32),
                                   thr_b, q, rho, i, _ptr(msb, ctypes.c_uint8), _ptr(v, ctypes.c_uint32),
                                   ctypes.byref(st))
    return msb, v


def mpc_match_lift(cfg: MpcCfg, g: Geom, mode: int, db_code, db_mask, q_code, q_mask, thr_b: int = 0,
                   want_z: bool = False):
    """Alg. 3 with ConstLift (code shares u16, mask shares u32) or NoLift (both u32)."""
    ct = np.uint32 if mode == LIFT_NONE else np.uint16
    db_code = np.ascontiguousarray(db_code, dtype=ct)
    q_code = np.ascontiguousarray(q_code, dtype=ct)
    db_mask = np.ascontiguousarray(db_mask, dtype=np.uint32)
    q_mask = np.ascontiguousarray(q_mask, dtype=np.uint32)
    s, Q = db_code.shape[1], q_code.shape[1]
    n = Q * g.R
    zc = np.zeros((3, n, s), ct) if want_z else None
    zm = np.zeros((3, n, s), np.uint32) if want_z else None
    bits = np.zeros((3, Q), np.uint8)
    st = Stats()
    vp = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
    lib().orc_mpc_match_lift(ctypes.byref(cfg), ctypes.byref(g), mode, thr_b, vp(db_code),
                             _ptr(db_mask, ctypes.c_uint32), s, vp(q_code), _ptr(q_mask, ctypes.c_uint32), Q,
                             vp(zc), _ptr(zm, ctypes.c_uint32), _ptr(bits, ctypes.c_uint8), ctypes.byref(st))
    return {"bits": bits, "z_code": zc, "z_mask": zm, "stats": st.as_dict()}


# ---- transcript hash (a test aid) ----

def mix64(z: int) -> int:
    """The SplitMix64 output function."""
    return int(lib().orc_mix64(z & 0xFFFFFFFFFFFFFFFF))


def transcript_hash(z_code, z_mask, bits) -> int:
    """Fingerprint of a request's A4 messages z_code, z_mask ([3][n][s], u16 or u32; z_mask None
    for protocol 1) and output bit components bits [3][Q]."""
    zc = np.ascontiguousarray(z_code)
    zm = None if z_mask is None else np.ascontiguousarray(z_mask)
    b = np.ascontiguousarray(bits, dtype=np.uint8)
    vp = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
    return int(lib().orc_transcript_hash(vp(zc), zc.dtype.itemsize, vp(zm), 0 if zm is None else zm.dtype.itemsize,
                                         zc.shape[1], zc.shape[2], _ptr(b, ctypes.c_uint8), b.shape[1]))
