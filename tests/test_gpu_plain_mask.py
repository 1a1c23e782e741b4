"""Protocol 1 on the GPU (Sec. 4, Alg. 2: shared codes, public masks) against the oracle.

The comparison kernel's 16-bit MSB against the oracle's element by element on every boundary
of the threshold, and the whole context path (plaintext ml GEMM, shared code dot, comparison,
OR tree) on both share encodings: bit components equal to the oracle's for the request's id,
distances equal to the plaintext ones, opened bits equal to Alg. 1's. Integers throughout, so
every comparison is exact.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import galois, lib, load_workload, make_ctx, plain_mask_u16, query_shares_gpu, torch_mod, u16

pytestmark = pytest.mark.gpu

REQ = 11


@pytest.fixture(scope="module")
def torch():
    t = torch_mod()
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def wl(torch):
    """1,500 rows in two 1,024-row chunks (the second ragged), 2 queries x 31 rotations."""
    w = synth.Workload("plain", s=1500, Q=2, planted=2, seed=0x9A52)
    dc, dm = w.db_bits()
    qc, qm = w.query_bits()
    match, ml, hd = oracle.plain_match(oracle.iris_geom(), qc, qm, dc, dm, distances=True)
    return dict(w=w, dc=dc, dm=dm, qc=qc, qm=qm, match=match, ml=ml, hd=hd)


def test_encode_plain_mask_matches_oracle(torch, wl):
    """ipc_encode_plain_mask gives the public mask operand of Alg. 2: element b of row r is mask
    bit b, the value the oracle's mask shares reconstruct to (Sec. 4.1.1). Also a code length
    that ends inside a 64-bit word (l = 136) and a single row."""
    w = wl["w"]
    _, om = oracle.encode_share(wl["dc"], wl["dm"], w.l, w.db_share_seed, 0)
    got = plain_mask_u16(wl["dm"], w.l)
    torch.cuda.synchronize()
    assert (u16(got) == oracle.reconstruct_u16(om)).all()
    rng = np.random.default_rng(0x9A54)
    bits = rng.integers(0, 2**63, (3, 3), dtype=np.int64).view(np.uint64)
    for n, l in ((3, 136), (1, 8)):
        _, om = oracle.encode_share(bits[:n], bits[:n], l, 0x1234, 1)
        got = plain_mask_u16(bits[:n], l)
        torch.cuda.synchronize()
        assert (u16(got) == oracle.reconstruct_u16(om)).all(), (n, l)


def _boundary_cases(rng, n):
    """(ml, dot) pairs on and around the threshold 4 dot = ml, plus the extremes."""
    ml = rng.integers(0, 12801, n)
    ml[:64] = np.arange(64)
    ml[64:70] = 12800
    q4 = ml // 4
    pick = rng.integers(0, 6, n)
    dot = np.select([pick == 0, pick == 1, pick == 2, pick == 3, pick == 4],
                    [q4 - 1, q4, q4 + 1, -ml, ml], default=rng.integers(-ml, ml + 1))
    return ml.astype(np.int64), np.clip(dot, -ml, ml).astype(np.int64)


def test_compare_plain_kernel_matches_oracle(torch):
    """ipc_compare_plain: every comparison's MSB components equal the oracle's, 2 columns x
    1,000 rows (32-row words, the last ragged), values on every side of the threshold."""
    ipc = lib()
    rng = np.random.default_rng(0x9A53)
    n_cols, n_rows, ldz = 2, 1000, 1000
    ml, dot = _boundary_cases(rng, n_cols * n_rows)
    ml, dot = ml.reshape(n_cols, n_rows), dot.reshape(n_cols, n_rows)
    a = rng.integers(0, 1 << 16, (2, n_cols, n_rows))
    shares = np.stack([a[0], a[1], (dot - a[0] - a[1]) & 0xFFFF]).astype(np.uint16)
    seeds = (0x1111, 0x2222, 0x3333)
    tags = np.array([(REQ, (0 << 5) | 3), (REQ, (1 << 5) | 7)], np.uint32)
    dz = torch.from_numpy(shares.view(np.int16).copy()).cuda()
    dml = torch.from_numpy(ml.astype(np.uint16).view(np.int16).copy()).cuda()
    dtags = torch.from_numpy(tags.view(np.int32).copy()).cuda()
    nb = (n_rows + 1023) // 1024
    roots = torch.zeros((3, n_cols, nb), dtype=torch.int32, device="cuda")
    msb = torch.zeros((3, n_cols, n_rows), dtype=torch.uint8, device="cuda")
    ipc.ipc_compare_plain([dz[j] for j in range(3)], dml, ldz, n_cols, n_rows, 0, dtags, seeds, 16384, 5, roots, nb,
                          msb, n_rows)
    torch.cuda.synchronize()
    ipc.ipc_status()
    got = msb.cpu().numpy()
    assert (oracle.reconstruct_bits(got) == (4 * dot > ml)).all()
    cfg = oracle.mpc_cfg(seeds, req=REQ)
    for c, (q, rho) in enumerate(((0, 3), (1, 7))):
        for r in range(n_rows):
            ref = oracle.mpc_compare_plain(cfg, shares[:, c, r], int(ml[c, r]), q, rho, r)
            assert (got[:, c, r] == ref).all(), (c, r)


@pytest.mark.parametrize("path", ["tc", "tcg"])
def test_context_plain_mask_matches_oracle(wl, torch, path):
    ipc = lib()
    w = wl["w"]
    gal = galois(path)
    ctx = make_ctx(w, path=path, keep=True, chunk_rows=1024, plain_mask=True)
    try:
        load_workload(ctx, w, chunk=700, galois_shares=gal, plain_mask=True)
        assert ipc.ipc_db_rows(ctx) == w.s
        qcode, _ = query_shares_gpu(w, wl["qc"], wl["qm"], galois_shares=gal)
        qmask = plain_mask_u16(wl["qm"], w.l)
        rid = ipc.submit_queries(ctx, [qcode[j] for j in range(3)], [qmask, None, None], w.Q, 1)
        sh = np.zeros((3, w.Q), np.uint8)
        ipc.fetch_bit_shares(ctx, rid, sh, w.Q, 60000)
        enc = oracle.encode_share_galois if gal else oracle.encode_share
        dbc, _ = enc(wl["dc"], wl["dm"], w.l, w.db_share_seed, 0)
        assert (u16(qcode) == enc(wl["qc"], wl["qm"], w.l, w.q_share_seed, 1)[0]).all()
        ref = oracle.mpc_match_plain(oracle.mpc_cfg(w.prf_seeds, req=rid), oracle.iris_geom(), dbc, wl["dm"],
                                     u16(qcode), wl["qm"], galois=gal, want_z=True)
        assert (sh == ref["bits"]).all()
        # protocol 1's messages: the code dot products and the output components (ml is public)
        assert ipc.fetch_transcript_hash(ctx, rid) == oracle.transcript_hash(ref["z_code"], None, ref["bits"])
        for q, rho in ((0, 0), (0, 15), (1, 30)):
            dot = np.zeros(w.s, np.int16)
            ml = np.zeros(w.s, np.uint16)
            ipc.fetch_distances(ctx, rid, q, rho, 0, w.s, dot, ml)
            assert (ml == wl["ml"][q, rho]).all()
            assert (dot == wl["ml"][q, rho] - 2 * wl["hd"][q, rho]).all()
        bits = np.zeros(w.Q, np.uint8)
        ipc.fetch_match_bits(ctx, rid, bits, w.Q, 60000)
        assert (bits == wl["match"]).all() and bits.sum() == w.planted
    finally:
        ipc.ipc_destroy(ctx)


def test_plain_mask_refusals(wl, torch):
    """Protocol 1 needs the tensor-core paths and a public mask; serving refuses it."""
    ipc = lib()
    w = wl["w"]
    with pytest.raises(ipc.IpcError):
        make_ctx(w, path="i8mma", plain_mask=True)
    ctx = make_ctx(w, path="tc", chunk_rows=1024, plain_mask=True)
    try:
        load_workload(ctx, w, chunk=1100, plain_mask=True)
        with pytest.raises(ipc.IpcError):
            ipc.ipc_serve_start(ctx, pool_queries=4, variant="tc256")
        qcode, _ = query_shares_gpu(w, wl["qc"], wl["qm"])
        with pytest.raises(ipc.IpcError):   # the public mask is required
            ipc.submit_queries(ctx, [qcode[j] for j in range(3)], [None, None, None], w.Q, 1)
    finally:
        ipc.ipc_destroy(ctx)
