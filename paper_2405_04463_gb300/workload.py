"""Loading a seeded synthetic workload into the library through its C ABI.

The database bits come from the seeded generator (synth, device half), the client-side
encoding and sharing (A0) from ipc_encode_share, and the resident planes (A1) from
load_db_shares. Used by the benchmark, the smoke check and the GPU tests."""
from __future__ import annotations

import numpy as np

import synth


def torch_mod():
    import torch
    return torch


def lib():
    from . import binding
    return binding


def dev_u64(a):
    torch = torch_mod()
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def galois(path) -> bool:
    """Whether a path takes Galois-ring Shamir shares (else replicated-sharing components)."""
    return path in ("tcg", 4)


def encode_gpu(code_bits, mask_bits, l, seed, side, idx0=0, galois_shares=False):
    """A0 on the device through the C ABI; returns torch int16 [3][n][l] code and mask shares
    (additive components, or the parties' Galois-ring Shamir shares)."""
    torch = torch_mod()
    ipc = lib()
    cb = code_bits if hasattr(code_bits, "data_ptr") else dev_u64(code_bits)
    mb = mask_bits if hasattr(mask_bits, "data_ptr") else dev_u64(mask_bits)
    n = cb.shape[0]
    code = torch.empty((3, n, l), dtype=torch.int16, device="cuda")
    mask = torch.empty((3, n, l), dtype=torch.int16, device="cuda")
    fn = ipc.ipc_encode_share_galois if galois_shares else ipc.ipc_encode_share
    fn(cb, mb, n, l, seed, side, idx0, code, mask)
    return code, mask


def encode_gpu32(code_bits, mask_bits, l, seed, side, idx0=0):
    """A0 over Z_2^32 through the C ABI: torch int32 [3][n][l] code and mask shares."""
    torch = torch_mod()
    ipc = lib()
    cb = code_bits if hasattr(code_bits, "data_ptr") else dev_u64(code_bits)
    mb = mask_bits if hasattr(mask_bits, "data_ptr") else dev_u64(mask_bits)
    n = cb.shape[0]
    code = torch.empty((3, n, l), dtype=torch.int32, device="cuda")
    mask = torch.empty((3, n, l), dtype=torch.int32, device="cuda")
    ipc.ipc_encode_share32(cb, mb, n, l, seed, side, idx0, code, mask)
    return code, mask


def lift_shares(code_bits, mask_bits, l, seed, side, idx0=0, lift="const"):
    """Shares of a lifting variant: ConstLift takes Z_2^16 code shares and Z_2^32 mask shares,
    NoLift Z_2^32 shares of both."""
    c32, m32 = encode_gpu32(code_bits, mask_bits, l, seed, side, idx0)
    if lift in ("none", 2):
        return c32, m32
    c16, _ = encode_gpu(code_bits, mask_bits, l, seed, side, idx0)
    return c16, m32


def u16(t) -> np.ndarray:
    """torch int16 tensor -> numpy uint16."""
    return t.cpu().numpy().view(np.uint16)


def tags_for(req: int, Q: int, R: int):
    t = np.zeros((Q * R, 2), np.uint32)
    for q in range(Q):
        for rho in range(R):
            t[q * R + rho] = (req, (q << 5) | rho)
    return t


def db_bits_device(w: synth.Workload, row0: int, n: int):
    """Database bits of rows row0..row0+n-1 generated on the device (synth device generator)."""
    torch = torch_mod()
    code = torch.empty((n, w.nwords), dtype=torch.int64, device="cuda")
    mask = torch.empty((n, w.nwords), dtype=torch.int64, device="cuda")
    synth.device_db_bits(w.seed, row0, n, w.l, code.data_ptr(), mask.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    return code, mask


def plain_mask_u16(mask_bits, l: int):
    """Packed mask bits [n][words] (numpy or device int64) -> device int16 [n][l] of 0/1 through
    ipc_encode_plain_mask: the public mask operand of protocol 1."""
    torch = torch_mod()
    mb = mask_bits if hasattr(mask_bits, "data_ptr") else dev_u64(mask_bits)
    out = torch.empty((mb.shape[0], l), dtype=torch.int16, device="cuda")
    lib().ipc_encode_plain_mask(mb, mb.shape[0], l, out)
    return out


def load_workload(ctx, w: synth.Workload, chunk: int = 16384, galois_shares=False, plain_mask=False, lift=None):
    """Generate the workload's database on the device, share it (A0) and load it (A1). With
    plain_mask the masks stay public (protocol 1): mask[0] carries the 0/1 mask elements."""
    torch = torch_mod()
    ipc = lib()
    for r0 in range(0, w.s, chunk):
        n = min(chunk, w.s - r0)
        cb, mb = db_bits_device(w, r0, n)
        if lift not in (None, "mpc", 0):
            code, mask = lift_shares(cb, mb, w.l, w.db_share_seed, 0, idx0=r0, lift=lift)
        else:
            code, mask = encode_gpu(cb, mb, w.l, w.db_share_seed, 0, idx0=r0, galois_shares=galois_shares)
        masks = [plain_mask_u16(mb, w.l), None, None] if plain_mask else [mask[j] for j in range(3)]
        ipc.load_db_shares(ctx, [code[j] for j in range(3)], masks, n, 1)
        del code, mask, masks
    torch.cuda.synchronize()


def query_shares_gpu(w: synth.Workload, qc=None, qm=None, galois_shares=False):
    if qc is None:
        qc, qm = w.query_bits()
    return encode_gpu(qc, qm, w.l, w.q_share_seed, 1, galois_shares=galois_shares)


def make_ctx(w: synth.Workload, path="i8mma", keep=False, chunk_rows=0, max_queries=0, plain_mask=False,
             lift="mpc", thr_b=0, max_requests=0, fused=False):
    ipc = lib()
    g = ipc.ipc_geom(w.rows, w.cols, w.cell, w.rot_lo, w.R)
    cfg = ipc.make_config(g, thr_a=w.thr_a, path=path, db_chunk_rows=chunk_rows, max_queries=max_queries or w.Q,
                          seeds=w.prf_seeds, keep_distances=keep, plain_mask=plain_mask, lift=lift, thr_b=thr_b,
                          max_requests=max_requests, fused=fused)
    ctx = ipc.ipc_create(cfg)
    ipc.ipc_set_input_stream(ctx)   # device inputs come from torch's current stream
    return ctx
