"""GB300-native share-domain iris uniqueness check (arXiv 2405.04463, Alg. 3 hot path).

Thin ctypes binding over the C ABI of ``libipcheck.so`` (declared in include/ipcheck.h).
Functions carry the C names and only marshal arguments: every step of the hot path runs
in the library's CUDA kernels. Pointer arguments accept torch tensors (their data_ptr),
numpy arrays (host memory) or plain integers. A non-zero return code raises IpcError.

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_2405_04463_gb300.build``); importing fails loudly otherwise -- there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libipcheck.so")

IPC_OK, IPC_EINVAL, IPC_ENOMEM, IPC_ECUDA, IPC_ETIMEOUT = 0, -1, -2, -3, -4
IPC_EAGAIN, IPC_ENOTFOUND, IPC_EDEVICE, IPC_ENOSYS = -5, -6, -7, -8
IPC_PATH_I8MMA, IPC_PATH_I32, IPC_PATH_I8MIX, IPC_PATH_TC, IPC_PATH_TCG = 0, 1, 2, 3, 4
PATHS = {"i8mma": IPC_PATH_I8MMA, "i32": IPC_PATH_I32, "i8mix": IPC_PATH_I8MIX, "tc": IPC_PATH_TC,
         "tcg": IPC_PATH_TCG}


class IpcError(RuntimeError):
    def __init__(self, rc: int, msg: str):
        super().__init__(f"ipcheck error {rc}: {msg}")
        self.rc = rc


class ipc_geom(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_uint32), ("cols", ctypes.c_uint32), ("cell", ctypes.c_uint32),
                ("rot_lo", ctypes.c_int32), ("R", ctypes.c_uint32)]

    @property
    def l(self) -> int:
        return self.rows * self.cols * self.cell


def iris_geom(rot_lo: int = -15, R: int = 31) -> ipc_geom:
    return ipc_geom(16, 200, 4, rot_lo, R)


class ipc_config(ctypes.Structure):
    _fields_ = [("geom", ipc_geom), ("thr_a", ctypes.c_uint32), ("path", ctypes.c_int32),
                ("db_chunk_rows", ctypes.c_uint32), ("max_queries", ctypes.c_uint32),
                ("seeds", ctypes.c_uint64 * 3), ("keep_distances", ctypes.c_uint32), ("device", ctypes.c_int32),
                ("plain_mask", ctypes.c_uint32), ("lift", ctypes.c_uint32), ("thr_b", ctypes.c_uint32),
                ("max_requests", ctypes.c_uint32), ("fused", ctypes.c_uint32)]


LIFTS = {"mpc": 0, "const": 1, "none": 2}


IPC_SERVE_AUTOTUNE = -1
SERVE_VARIANTS = {"tc256": 0, "tc128": 1, "mix128": 0, "mma128": 1, "mma64": 2, "mma32": 3}


class ipc_serve_config(ctypes.Structure):
    _fields_ = [("pool_queries", ctypes.c_uint32), ("max_pending", ctypes.c_uint32), ("variant", ctypes.c_int32),
                ("tune_cache", ctypes.c_char_p)]


class ipc_serve_counters(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint64), ("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("pending", ctypes.c_uint64), ("comparisons", ctypes.c_double), ("elapsed_s", ctypes.c_double),
                ("pool_queries", ctypes.c_uint32), ("pool_cols", ctypes.c_uint32), ("n_chunks", ctypes.c_uint32),
                ("variant_steps", ctypes.c_uint64 * 4)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first (__graft_entry__.build()); "
                      "there is no CPU fallback")

lib = ctypes.CDLL(LIB_PATH)

_vp, _u8, _u16, _u32, _u64, _i32 = (ctypes.c_void_p, ctypes.c_uint8, ctypes.c_uint16, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_int32)
_sz, _int = ctypes.c_size_t, ctypes.c_int
_VP2, _VP3, _U64x3 = _vp * 2, _vp * 3, _u64 * 3
_VP4, _VP8 = _vp * 4, _vp * 8

_SIGS = {
    "ipc_encode_share": [_vp, _vp, _u32, _u32, _u64, _u32, _u32, _vp, _vp, _vp],
    "ipc_encode_plain_mask": [_vp, _u32, _u32, _vp, _vp],
    "ipc_split_limbs": [_vp, _sz, _vp, _vp, _vp],
    "ipc_prep_query": [_vp, _u32, ctypes.POINTER(ipc_geom), _u32, _vp, _vp, _u32, _vp],
    "ipc_encode_share32": [_vp, _vp, _u32, _u32, _u64, _u32, _u32, _vp, _vp, _vp],
    "ipc_split_limbs32": [_vp, _sz, _VP4, _vp],
    "ipc_prep_query32_f16": [_vp, _u32, ctypes.POINTER(ipc_geom), _u32, _u32, _VP4, _u32, _vp],
    "ipc_ring_gemm_tc32": [_u32, _VP8, _sz, _VP4, _u32, _u32, _u32, _vp, _u64, _u64, _u32, _vp, _sz, _u64, _vp],
    "ipc_compare_liftfree": [_vp, _vp, _VP3, _sz, _u32, _sz, _u64, _vp, _U64x3, _u32, _u32, _u32, _vp, _sz, _vp,
                             _sz, _vp],
    "ipc_encode_share_galois": [_vp, _vp, _u32, _u32, _u64, _u32, _u32, _vp, _vp, _vp],
    "ipc_prep_query_galois": [_vp, _u32, ctypes.POINTER(ipc_geom), _u32, _vp, _vp, _u32, _vp],
    "ipc_ring_gemm_tc_galois": [_u32, _vp, _vp, _sz, _vp, _vp, _u32, _u32, _u32, _vp, _u64, _u64, _u32, _vp, _sz,
                                _u64, _vp, _vp, _vp],
    "ipc_prep_query_f16": [_vp, _u32, ctypes.POINTER(ipc_geom), _u32, _vp, _vp, _u32, _vp],
    "ipc_ring_gemm_tc": [_VP2, _VP2, _sz, _vp, _vp, _u32, _u32, _u32, _vp, _u64, _u64, _u32, _vp, _sz, _u64, _vp],
    "ipc_ring_gemm_tc_tiles": [_u32, _VP2, _VP2, _sz, _vp, _vp, _u32, _u32, _u32, _vp, _u64, _u64, _u32, _vp, _sz,
                               _u64, _vp, _vp, _vp],
    "ipc_ring_gemm": [_int, _VP2, _VP2, _sz, _vp, _vp, _u32, _u32, _u32, _vp, _u64, _u64, _u32, _vp, _sz, _u64, _vp],
    "ipc_ring_gemm_tiles": [_int, _VP2, _VP2, _sz, _vp, _vp, _u32, _u32, _u32, _vp, _u64, _u64, _u32, _vp, _sz,
                            _u64, _vp, _vp, _vp],
    "ipc_compare": [_VP3, _VP3, _sz, _u32, _sz, _u64, _vp, _U64x3, _u32, _u32, _vp, _sz, _vp, _sz, _vp],
    "ipc_compare_plain": [_VP3, _vp, _sz, _u32, _sz, _u64, _vp, _U64x3, _u32, _u32, _vp, _sz, _vp, _sz, _vp],
    "ipc_or_finalize": [_vp, _sz, _u32, _u32, _u32, _u32, _vp, _U64x3, _vp, _vp],
    "ipc_status": [],
    "ipc_compare_or_noalloc": [_VP3, _VP3, _sz, _u32, _u32, _sz, _vp, _U64x3, _u32, _vp, _vp],
    "ipc_create": [ctypes.POINTER(ipc_config), ctypes.POINTER(_vp)],
    "load_db_shares": [_vp, _VP3, _VP3, _sz, _int],
    "submit_queries": [_vp, _VP3, _VP3, _sz, _int, ctypes.POINTER(_u64)],
    "fetch_match_bits": [_vp, _u64, _vp, _sz, _int],
    "fetch_bit_shares": [_vp, _u64, _vp, _sz, _int],
    "fetch_distances": [_vp, _u64, _u32, _u32, _sz, _sz, _vp, _vp],
    "fetch_transcript_hash": [_vp, _u64, ctypes.POINTER(_u64), _int],
    "ipc_selftest_bounded_wait": [_u32, _vp],
    "ipc_release": [_vp, _u64],
    "ipc_debug_stall_party": [_vp, _u32, _u32],
    "ipc_db_rows": [_vp],
    "ipc_destroy": [_vp],
    "ipc_last_error": [_vp],
    "ipc_ctx_stream": [_vp],
    "ipc_set_input_stream": [_vp, _vp],
    "ipc_measure_peak": [_int, _vp, ctypes.POINTER(ctypes.c_double)],
    "ipc_check_persons": [_vp * 2, _vp * 6, _vp * 6, _u32, _int, _vp, _vp, _int],
    "ipc_serve_start": [_vp, ctypes.POINTER(ipc_serve_config)],
    "ipc_serve_submit": [_vp, _VP3, _VP3, _sz, ctypes.POINTER(_u64)],
    "ipc_serve_stop": [_vp],
    "ipc_serve_stats": [_vp, ctypes.POINTER(ipc_serve_counters)],
    "ipc_serve_times": [_vp, _u64, ctypes.POINTER(ctypes.c_double)],
    "ipc_serve_tuning": [_vp, ctypes.c_char_p, _sz],
    "ipc_serve_tile_list": [_vp, _vp, _u32, _u32, _vp, _u32],
    "ipc_serve_first_fit": [_vp, _u32, _u32],
}
for _name, _args in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _int
lib.ipc_destroy.restype = None
lib.ipc_db_rows.restype = _sz
lib.ipc_last_error.restype = ctypes.c_char_p
lib.ipc_ctx_stream.restype = _vp
lib.ipc_serve_first_fit.restype = ctypes.c_int64


def ptr(x) -> int | None:
    """Address of a torch tensor, numpy array or integer (None stays None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s) -> int | None:
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(rc: int, ctx=None):
    if rc != IPC_OK:
        msg = lib.ipc_last_error(ctx)
        raise IpcError(rc, msg.decode() if msg else "")


# ---------------------------------------------------------------------------------------------
# Stage-level entry points
# ---------------------------------------------------------------------------------------------

def ipc_encode_share(code_bits, mask_bits, n, l, client_seed, side, idx0, code_sh, mask_sh, stream=None):
    _check(lib.ipc_encode_share(ptr(code_bits), ptr(mask_bits), n, l, client_seed & (2**64 - 1), side, idx0,
                                ptr(code_sh), ptr(mask_sh), _stream(stream)))


def ipc_encode_plain_mask(mask_bits, n, l, mask_out, stream=None):
    _check(lib.ipc_encode_plain_mask(ptr(mask_bits), n, l, ptr(mask_out), _stream(stream)))


def ipc_split_limbs(x, count, lo, hi, stream=None):
    _check(lib.ipc_split_limbs(ptr(x), count, ptr(lo), ptr(hi), _stream(stream)))


def ipc_prep_query(y, Q, geom: ipc_geom, party, b_lo, b_hi, n_pad, stream=None):
    _check(lib.ipc_prep_query(ptr(y), Q, ctypes.byref(geom), party, ptr(b_lo), ptr(b_hi), n_pad, _stream(stream)))


def ipc_ring_gemm(path, x_lo, x_hi, x_rows, b_lo, b_hi, n_cols, n_pad, l, col_tags, seed_own, seed_prev, vec, z,
                  ldz, row0, stream=None):
    path = PATHS.get(path, path)
    _check(lib.ipc_ring_gemm(path, _VP2(*[ptr(a) for a in x_lo]), _VP2(*[ptr(a) for a in x_hi]), x_rows, ptr(b_lo),
                             ptr(b_hi), n_cols, n_pad, l, ptr(col_tags), seed_own & (2**64 - 1),
                             seed_prev & (2**64 - 1), vec, ptr(z), ldz, row0, _stream(stream)))


def ipc_prep_query_f16(y, Q, geom: ipc_geom, party, b_lo, b_hi, n_pad, stream=None):
    _check(lib.ipc_prep_query_f16(ptr(y), Q, ctypes.byref(geom), party, ptr(b_lo), ptr(b_hi), n_pad,
                                  _stream(stream)))


def ipc_encode_share32(code_bits, mask_bits, n, l, client_seed, side, idx0, code_sh, mask_sh, stream=None):
    _check(lib.ipc_encode_share32(ptr(code_bits), ptr(mask_bits), n, l, client_seed & (2**64 - 1), side, idx0,
                                  ptr(code_sh), ptr(mask_sh), _stream(stream)))


def ipc_split_limbs32(x, count, limbs, stream=None):
    _check(lib.ipc_split_limbs32(ptr(x), count, _VP4(*[ptr(a) for a in limbs]), _stream(stream)))


def ipc_prep_query32_f16(y, Q, geom: ipc_geom, party, segments, b, n_pad, stream=None):
    _check(lib.ipc_prep_query32_f16(ptr(y), Q, ctypes.byref(geom), party, segments, _VP4(*[ptr(a) for a in b]),
                                    n_pad, _stream(stream)))


def ipc_ring_gemm_tc32(segments, x, x_rows, b, n_cols, n_pad, l, col_tags, seed_own, seed_prev, vec, z, ldz, row0,
                       stream=None):
    xs = list(x) + [None] * (8 - len(x))
    _check(lib.ipc_ring_gemm_tc32(segments, _VP8(*[ptr(a) for a in xs]), x_rows, _VP4(*[ptr(a) for a in b]), n_cols,
                                  n_pad, l, ptr(col_tags), seed_own & (2**64 - 1), seed_prev & (2**64 - 1), vec,
                                  ptr(z), ldz, row0, _stream(stream)))


def ipc_compare_liftfree(z16, z32, ml32, ldz, n_cols, n_rows, row0, col_tags, seeds, thr_a, thr_b,
                         log2_block_words, roots, ld_roots, msb_out=None, ld_msb=0, stream=None):
    p3 = lambda v: None if v is None else ctypes.cast(_VP3(*[ptr(a) for a in v]), _vp)
    _check(lib.ipc_compare_liftfree(p3(z16), p3(z32), _VP3(*[ptr(a) for a in ml32]), ldz, n_cols, n_rows, row0, ptr(col_tags),
                                    _U64x3(*[s & (2**64 - 1) for s in seeds]), thr_a, thr_b, log2_block_words,
                                    ptr(roots), ld_roots, ptr(msb_out), ld_msb, _stream(stream)))


def ipc_encode_share_galois(code_bits, mask_bits, n, l, client_seed, side, idx0, code_sh, mask_sh, stream=None):
    _check(lib.ipc_encode_share_galois(ptr(code_bits), ptr(mask_bits), n, l, client_seed & (2**64 - 1), side, idx0,
                                       ptr(code_sh), ptr(mask_sh), _stream(stream)))


def ipc_prep_query_galois(y, Q, geom: ipc_geom, party, b_lo, b_hi, n_pad, stream=None):
    _check(lib.ipc_prep_query_galois(ptr(y), Q, ctypes.byref(geom), party, ptr(b_lo), ptr(b_hi), n_pad,
                                     _stream(stream)))


def ipc_ring_gemm_tc_galois(tile_cols, x_lo, x_hi, x_rows, b_lo, b_hi, n_cols, n_pad, l, col_tags, seed_own,
                            seed_prev, vec, z, ldz, row0, col_tiles=None, n_col_list=None, stream=None):
    _check(lib.ipc_ring_gemm_tc_galois(tile_cols, ptr(x_lo), ptr(x_hi), x_rows, ptr(b_lo), ptr(b_hi), n_cols, n_pad, l,
                                       ptr(col_tags), seed_own & (2**64 - 1), seed_prev & (2**64 - 1), vec, ptr(z),
                                       ldz, row0, ptr(col_tiles), ptr(n_col_list), _stream(stream)))


def ipc_ring_gemm_tc(x_lo, x_hi, x_rows, b_lo, b_hi, n_cols, n_pad, l, col_tags, seed_own, seed_prev, vec, z, ldz,
                     row0, stream=None):
    _check(lib.ipc_ring_gemm_tc(_VP2(*[ptr(a) for a in x_lo]), _VP2(*[ptr(a) for a in x_hi]), x_rows, ptr(b_lo),
                                ptr(b_hi), n_cols, n_pad, l, ptr(col_tags), seed_own & (2**64 - 1),
                                seed_prev & (2**64 - 1), vec, ptr(z), ldz, row0, _stream(stream)))


def ipc_ring_gemm_tc_tiles(tile_cols, x_lo, x_hi, x_rows, b_lo, b_hi, n_cols, n_pad, l, col_tags, seed_own,
                           seed_prev, vec, z, ldz, row0, col_tiles=None, n_col_list=None, stream=None):
    _check(lib.ipc_ring_gemm_tc_tiles(tile_cols, _VP2(*[ptr(a) for a in x_lo]), _VP2(*[ptr(a) for a in x_hi]),
                                      x_rows, ptr(b_lo), ptr(b_hi), n_cols, n_pad, l, ptr(col_tags),
                                      seed_own & (2**64 - 1), seed_prev & (2**64 - 1), vec, ptr(z), ldz, row0,
                                      ptr(col_tiles), ptr(n_col_list), _stream(stream)))


IPC_GEMM_MIX128, IPC_GEMM_MMA128, IPC_GEMM_MMA64, IPC_GEMM_MMA32 = 0, 1, 2, 3


def ipc_ring_gemm_tiles(variant, x_lo, x_hi, x_rows, b_lo, b_hi, n_cols, n_pad, l, col_tags, seed_own, seed_prev,
                        vec, z, ldz, row0, col_tiles=None, n_col_list=None, stream=None):
    _check(lib.ipc_ring_gemm_tiles(variant, _VP2(*[ptr(a) for a in x_lo]), _VP2(*[ptr(a) for a in x_hi]), x_rows,
                                   ptr(b_lo), ptr(b_hi), n_cols, n_pad, l, ptr(col_tags), seed_own & (2**64 - 1),
                                   seed_prev & (2**64 - 1), vec, ptr(z), ldz, row0, ptr(col_tiles),
                                   ptr(n_col_list), _stream(stream)))


def ipc_compare(z_code, z_mask, ldz, n_cols, n_rows, row0, col_tags, seeds, thr_a, log2_block_words, roots,
                ld_roots, msb_out=None, ld_msb=0, stream=None):
    _check(lib.ipc_compare(_VP3(*[ptr(a) for a in z_code]), _VP3(*[ptr(a) for a in z_mask]), ldz, n_cols, n_rows,
                           row0, ptr(col_tags), _U64x3(*[s & (2**64 - 1) for s in seeds]), thr_a, log2_block_words,
                           ptr(roots), ld_roots, ptr(msb_out), ld_msb, _stream(stream)))


def ipc_compare_plain(z_code, ml, ldz, n_cols, n_rows, row0, col_tags, seeds, thr_a, log2_block_words, roots,
                      ld_roots, msb_out=None, ld_msb=0, stream=None):
    _check(lib.ipc_compare_plain(_VP3(*[ptr(a) for a in z_code]), ptr(ml), ldz, n_cols, n_rows, row0, ptr(col_tags),
                                 _U64x3(*[s & (2**64 - 1) for s in seeds]), thr_a, log2_block_words, ptr(roots),
                                 ld_roots, ptr(msb_out), ld_msb, _stream(stream)))


def ipc_or_finalize(roots, ld_roots, n_blocks, log2_block_words, Q, R, col_tags, seeds, bit_shares, stream=None):
    _check(lib.ipc_or_finalize(ptr(roots), ld_roots, n_blocks, log2_block_words, Q, R, ptr(col_tags),
                               _U64x3(*[s & (2**64 - 1) for s in seeds]), ptr(bit_shares), _stream(stream)))


def ipc_compare_or_noalloc(z_code, z_mask, ldz, Q, R, n_rows, col_tags, seeds, thr_a, bit_shares, stream=None):
    _check(lib.ipc_compare_or_noalloc(_VP3(*[ptr(a) for a in z_code]), _VP3(*[ptr(a) for a in z_mask]), ldz, Q, R,
                                      n_rows, ptr(col_tags), _U64x3(*[s & (2**64 - 1) for s in seeds]), thr_a,
                                      ptr(bit_shares), _stream(stream)))


def ipc_status():
    _check(lib.ipc_status())


def ipc_selftest_bounded_wait(limit_us, stream=None):
    _check(lib.ipc_selftest_bounded_wait(limit_us, _stream(stream)))


# ---------------------------------------------------------------------------------------------
# Context-level API
# ---------------------------------------------------------------------------------------------

def make_config(geom: ipc_geom | None = None, thr_a: int = 16384, path="i8mma", db_chunk_rows: int = 0,
                max_queries: int = 0, seeds=(0x51EED0, 0x51EED1, 0x51EED2), keep_distances: bool = False,
                device: int = 0, plain_mask: bool = False, lift="mpc", thr_b: int = 0,
                max_requests: int = 0, fused: bool = False) -> ipc_config:
    c = ipc_config()
    c.geom = geom if geom is not None else iris_geom()
    c.thr_a = thr_a
    c.path = PATHS.get(path, path)
    c.db_chunk_rows = db_chunk_rows
    c.max_queries = max_queries
    for j in range(3):
        c.seeds[j] = seeds[j] & (2**64 - 1)
    c.keep_distances = 1 if keep_distances else 0
    c.device = device
    c.plain_mask = 1 if plain_mask else 0
    c.lift = LIFTS.get(lift, lift)
    c.thr_b = thr_b
    c.max_requests = max_requests
    c.fused = 1 if fused else 0
    return c


def ipc_create(cfg: ipc_config) -> int:
    h = _vp()
    _check(lib.ipc_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def load_db_shares(ctx, code, mask, n_rows, src_is_device):
    _check(lib.load_db_shares(ctx, _VP3(*[ptr(a) for a in code]), _VP3(*[ptr(a) for a in mask]), n_rows,
                              1 if src_is_device else 0), ctx)


def submit_queries(ctx, code, mask, n_queries, src_is_device) -> int:
    rid = _u64()
    _check(lib.submit_queries(ctx, _VP3(*[ptr(a) for a in code]), _VP3(*[ptr(a) for a in mask]), n_queries,
                              1 if src_is_device else 0, ctypes.byref(rid)), ctx)
    return rid.value


def fetch_transcript_hash(ctx, req_id, timeout_ms=-1) -> int:
    h = _u64()
    _check(lib.fetch_transcript_hash(ctx, req_id, ctypes.byref(h), timeout_ms), ctx)
    return h.value


def fetch_match_bits(ctx, req_id, bits_out, n_queries, timeout_ms=-1):
    _check(lib.fetch_match_bits(ctx, req_id, ptr(bits_out), n_queries, timeout_ms), ctx)


def fetch_bit_shares(ctx, req_id, shares_out, n_queries, timeout_ms=-1):
    _check(lib.fetch_bit_shares(ctx, req_id, ptr(shares_out), n_queries, timeout_ms), ctx)


def fetch_distances(ctx, req_id, q, rho, row_begin, row_end, dot, ml):
    _check(lib.fetch_distances(ctx, req_id, q, rho, row_begin, row_end, ptr(dot), ptr(ml)), ctx)


def ipc_debug_stall_party(ctx, party, limit_us):
    _check(lib.ipc_debug_stall_party(ctx, party, limit_us), ctx)


def ipc_release(ctx, req_id):
    _check(lib.ipc_release(ctx, req_id), ctx)


def ipc_db_rows(ctx) -> int:
    return lib.ipc_db_rows(ctx)


def ipc_destroy(ctx):
    lib.ipc_destroy(ctx)


def ipc_set_input_stream(ctx, stream=None):
    _check(lib.ipc_set_input_stream(ctx, _stream(stream)), ctx)


def ipc_ctx_stream(ctx) -> int:
    return lib.ipc_ctx_stream(ctx) or 0


def ipc_measure_peak(what: int, stream=None) -> float:
    out = ctypes.c_double()
    _check(lib.ipc_measure_peak(what, _stream(stream), ctypes.byref(out)))
    return out.value


def ipc_last_error(ctx=None) -> str:
    m = lib.ipc_last_error(ctx)
    return m.decode() if m else ""


# ---------------------------------------------------------------------------------------------
# Serving (continuous batching)
# ---------------------------------------------------------------------------------------------

def ipc_serve_start(ctx, pool_queries: int = 0, max_pending: int = 0, variant=IPC_SERVE_AUTOTUNE,
                    tune_cache: str | None = None):
    v = SERVE_VARIANTS.get(variant, variant)
    cfg = ipc_serve_config(pool_queries, max_pending, v, tune_cache.encode() if tune_cache else None)
    _check(lib.ipc_serve_start(ctx, ctypes.byref(cfg)), ctx)


def ipc_serve_submit(ctx, code, mask, n_queries) -> int:
    """code[j], mask[j]: host arrays (numpy or pinned CPU tensors) [n_queries][l] uint16/int16."""
    rid = _u64(0)
    _check(lib.ipc_serve_submit(ctx, _VP3(*[ptr(a) for a in code]), _VP3(*[ptr(a) for a in mask]), n_queries,
                                ctypes.byref(rid)), ctx)
    return rid.value


def ipc_serve_stop(ctx):
    _check(lib.ipc_serve_stop(ctx), ctx)


def ipc_serve_stats(ctx) -> dict:
    out = ipc_serve_counters()
    _check(lib.ipc_serve_stats(ctx, ctypes.byref(out)), ctx)
    return {"steps": out.steps, "admitted": out.admitted, "completed": out.completed, "pending": out.pending,
            "comparisons": out.comparisons, "elapsed_s": out.elapsed_s, "pool_queries": out.pool_queries,
            "pool_cols": out.pool_cols, "n_chunks": out.n_chunks, "variant_steps": list(out.variant_steps)}


def ipc_serve_times(ctx, req_id) -> tuple:
    out = (ctypes.c_double * 3)()
    _check(lib.ipc_serve_times(ctx, req_id, out), ctx)
    return tuple(out)


def ipc_serve_tuning(ctx) -> str:
    buf = ctypes.create_string_buffer(1 << 16)
    _check(lib.ipc_serve_tuning(ctx, buf, len(buf)), ctx)
    return buf.value.decode()


def ipc_serve_tile_list(col0, ncols, tile_cols):
    import numpy as np
    col0 = np.ascontiguousarray(col0, dtype=np.uint32)
    ncols = np.ascontiguousarray(ncols, dtype=np.uint32)
    cap = int(sum((c + n + tile_cols - 1) // tile_cols - c // tile_cols for c, n in zip(col0, ncols))) + 1
    out = np.zeros(cap, np.uint32)
    n = lib.ipc_serve_tile_list(ptr(col0), ptr(ncols), len(col0), tile_cols, ptr(out), cap)
    if n < 0:
        _check(n)
    return out[:n]


def ipc_serve_first_fit(used, want) -> int:
    import numpy as np
    used = np.ascontiguousarray(used, dtype=np.uint8)
    return int(lib.ipc_serve_first_fit(ptr(used), len(used), want))


# ---------------------------------------------------------------------------------------------
# Both eyes and inner-batch matching
# ---------------------------------------------------------------------------------------------

def ipc_check_persons(ctx_eyes, code, mask, P, src_is_device, timeout_ms=-1):
    """ctx_eyes: the two eyes' contexts; code, mask: 6 arrays each (eye-major, 3 components per
    eye) [P][l] uint16. Returns (bit components [3][P] uint8, request ids of the 5 parts)."""
    import numpy as np
    out = np.zeros((3, P), np.uint8)
    ids = (_u64 * 5)()
    _check(lib.ipc_check_persons((_vp * 2)(*ctx_eyes), (_vp * 6)(*[ptr(a) for a in code]),
                                 (_vp * 6)(*[ptr(a) for a in mask]), P, src_is_device, ptr(out),
                                 ctypes.cast(ids, _vp), timeout_ms), ctx_eyes[0])
    return out, list(ids)
