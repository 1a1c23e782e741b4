"""GPU parity: every stage of the CUDA path against the CPU oracle, through the C ABI.

Integers throughout, so every comparison is bit-exact: shares where both sides follow the
same PRF counter layout, reconstructions and opened bits otherwise.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import (db_bits_device, dev_u64, encode_gpu, lib, load_workload, make_ctx, query_shares_gpu,
                        tags_for, torch_mod, u16)

pytestmark = pytest.mark.gpu

L = 12800
REQ = 7


@pytest.fixture(scope="module")
def torch():
    t = torch_mod()
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def small(torch):
    """s = 777 rows (ragged against 128-row tiles and 32-row words), 5 queries x 31 rotations
    (155 columns: two 128-column tiles, the second ragged), 2 planted near-duplicates."""
    w = synth.Workload("small", s=777, Q=5, planted=2, seed=0xA11CE)
    dc, dm = w.db_bits()
    qc, qm = w.query_bits()
    dbc, dbm = oracle.encode_share(dc, dm, L, w.db_share_seed, 0)
    qsc, qsm = oracle.encode_share(qc, qm, L, w.q_share_seed, 1)
    ref = oracle.mpc_match(oracle.mpc_cfg(w.prf_seeds, req=REQ), oracle.iris_geom(), dbc, dbm, qsc, qsm,
                           want_z=True, want_msb=True)
    match, ml, hd = oracle.plain_match(oracle.iris_geom(), qc, qm, dc, dm, distances=True)
    return dict(w=w, dc=dc, dm=dm, qc=qc, qm=qm, dbc=dbc, dbm=dbm, qsc=qsc, qsm=qsm, ref=ref, match=match, ml=ml,
                hd=hd)


def test_split_limbs_exhaustive(torch):
    ipc = lib()
    x = torch.arange(65536, dtype=torch.int32).to(torch.int16).cuda()
    lo = torch.empty(65536, dtype=torch.int8, device="cuda")
    hi = torch.empty(65536, dtype=torch.int8, device="cuda")
    ipc.ipc_split_limbs(x, 65536, lo, hi)
    lo_, hi_ = lo.cpu().numpy().astype(np.int64), hi.cpu().numpy().astype(np.int64)
    assert ((256 * hi_ + lo_) & 0xFFFF == np.arange(65536)).all()
    assert lo_.min() >= -128 and lo_.max() <= 127 and hi_.min() >= -128 and hi_.max() <= 127


def test_prep_query_f16_is_the_int8_operand(small, torch):
    """The tcgen05 path's query operand is the int8 operand of ipc_prep_query, each limb as the
    fp16 pattern of its integer value, exactly (every row, padding rows included)."""
    ipc = lib()
    g = ipc.iris_geom()
    y = torch.from_numpy(small["qsc"].view(np.int16).copy()).cuda()
    n_pad = 256
    for party in range(3):
        lo8 = torch.empty((n_pad, 2 * L), dtype=torch.int8, device="cuda")
        hi8 = torch.empty((n_pad, 2 * L), dtype=torch.int8, device="cuda")
        ipc.ipc_prep_query(y, 5, g, party, lo8, hi8, n_pad)
        lo = torch.empty((n_pad, 2 * L), dtype=torch.int16, device="cuda")
        hi = torch.empty((n_pad, 2 * L), dtype=torch.int16, device="cuda")
        ipc.ipc_prep_query_f16(y, 5, g, party, lo, hi, n_pad)
        assert (lo.view(torch.float16).float() == lo8.float()).all()
        assert (hi.view(torch.float16).float() == hi8.float()).all()


def test_encode_share_matches_oracle(small):
    code, mask = encode_gpu(small["dc"], small["dm"], L, small["w"].db_share_seed, 0)
    assert (u16(code) == small["dbc"]).all()
    assert (u16(mask) == small["dbm"]).all()
    qcode, qmask = encode_gpu(small["qc"], small["qm"], L, small["w"].q_share_seed, 1)
    assert (u16(qcode) == small["qsc"]).all()
    assert (u16(qmask) == small["qsm"]).all()


def test_device_generator_matches_host(torch):
    w = synth.workload("c2")
    rows = np.array([0, 1, 31, 4097, 99_999])
    hc, hm = w.db_bits(rows)
    for k, r in enumerate(rows):
        c, m = db_bits_device(w, int(r), 1)
        assert (c.cpu().numpy().view(np.uint64)[0] == hc[k]).all()
        assert (m.cpu().numpy().view(np.uint64)[0] == hm[k]).all()


def test_prep_query_is_rotated_aby3_operand(small, torch):
    ipc = lib()
    g = ipc.iris_geom()
    og = oracle.iris_geom()
    Q, R = 5, 31
    y = torch.from_numpy(small["qsc"].view(np.int16).copy()).cuda()
    n_pad = 256
    for party in range(3):
        lo = torch.empty((n_pad, 2 * L), dtype=torch.int8, device="cuda")
        hi = torch.empty((n_pad, 2 * L), dtype=torch.int8, device="cuda")
        ipc.ipc_prep_query(y, Q, g, party, lo, hi, n_pad)
        rebuilt = (256 * hi.cpu().numpy().astype(np.int64) + lo.cpu().numpy().astype(np.int64)) & 0xFFFF
        prev = (party + 2) % 3
        for q in (0, 4):
            for rho in (0, 15, 30):
                ys = (small["qsc"][party, q].astype(np.uint32) + small["qsc"][prev, q]).astype(np.uint16)
                exp0 = oracle.rotate_u16(og, ys, -15 + rho)
                exp1 = oracle.rotate_u16(og, small["qsc"][party, q], -15 + rho)
                assert (rebuilt[q * R + rho, :L] == exp0).all()
                assert (rebuilt[q * R + rho, L:] == exp1).all()
        assert (rebuilt[Q * R:] == 0).all()


def _planes(torch, shares):
    """[3][n][l] uint16 numpy -> per component (lo, hi) device int8 limb planes via the C ABI (the
    resident database layout of every path)."""
    ipc = lib()
    out = []
    for j in range(3):
        x = torch.from_numpy(shares[j].view(np.int16).copy()).cuda()
        lo = torch.empty(x.shape, dtype=torch.int8, device="cuda")
        hi = torch.empty(x.shape, dtype=torch.int8, device="cuda")
        ipc.ipc_split_limbs(x, x.numel(), lo, hi)
        out.append((lo, hi))
    return out


def _gemm_all(torch, small, path):
    """A1-A3 for all parties and both vectors; returns z[vec] as numpy [3][N][s] uint16."""
    ipc = lib()
    g = ipc.iris_geom()
    w = small["w"]
    Q, R, s = w.Q, w.R, w.s
    N, n_pad = Q * R, 256
    tags = torch.from_numpy(tags_for(REQ, Q, R).view(np.int32)).cuda()
    ldz = 784
    out = []
    tc = path == "tc"
    for vec, (db, qs) in enumerate(((small["dbc"], small["qsc"]), (small["dbm"], small["qsm"]))):
        planes = _planes(torch, db)
        y = torch.from_numpy(qs.view(np.int16).copy()).cuda()
        z = torch.zeros((3, N, ldz), dtype=torch.int16, device="cuda")
        for i in range(3):
            prev = (i + 2) % 3
            blo = torch.empty((n_pad, 2 * L), dtype=torch.int16 if tc else torch.int8, device="cuda")
            bhi = torch.empty((n_pad, 2 * L), dtype=torch.int16 if tc else torch.int8, device="cuda")
            (ipc.ipc_prep_query_f16 if tc else ipc.ipc_prep_query)(y, Q, g, i, blo, bhi, n_pad)
            xl, xh = [planes[i][0], planes[prev][0]], [planes[i][1], planes[prev][1]]
            if tc:
                ipc.ipc_ring_gemm_tc(xl, xh, s, blo, bhi, N, n_pad, L, tags, w.prf_seeds[i], w.prf_seeds[prev], vec,
                                     z[i], ldz, 0)
            else:
                ipc.ipc_ring_gemm(path, xl, xh, s, blo, bhi, N, n_pad, L, tags, w.prf_seeds[i], w.prf_seeds[prev],
                                  vec, z[i], ldz, 0)
        torch.cuda.synchronize()
        ipc.ipc_status()
        out.append(u16(z)[:, :, :s])
    return out


@pytest.mark.parametrize("path", ["i8mma", "i8mix", "i32", "tc"])
def test_ring_gemm_matches_oracle_shares(small, torch, path):
    zc, zm = _gemm_all(torch, small, path)
    assert (zc == small["ref"]["z_code"]).all()
    assert (zm == small["ref"]["z_mask"]).all()
    # reconstructions are the plaintext dot products (App. B): dot = ml - 2 hd, ml
    n = small["w"].Q * small["w"].R
    assert (oracle.reconstruct_u16(zc) == ((small["ml"] - 2 * small["hd"]).reshape(n, -1) & 0xFFFF)).all()
    assert (oracle.reconstruct_u16(zm) == small["ml"].reshape(n, -1)).all()


def test_compare_and_or_tree_match_oracle_shares(small, torch):
    ipc = lib()
    w = small["w"]
    Q, R, s = w.Q, w.R, w.s
    N = Q * R
    ldz = 784
    tags = torch.from_numpy(tags_for(REQ, Q, R).view(np.int32)).cuda()
    zc = torch.zeros((3, N, ldz), dtype=torch.int16, device="cuda")
    zm = torch.zeros((3, N, ldz), dtype=torch.int16, device="cuda")
    zc[:, :, :s] = torch.from_numpy(small["ref"]["z_code"].view(np.int16).copy()).cuda()
    zm[:, :, :s] = torch.from_numpy(small["ref"]["z_mask"].view(np.int16).copy()).cuda()
    for p in (0, 2, 5):  # block sizes 1, 4, 32 words give the same tree
        nb = (s + (32 << p) - 1) >> (5 + p)
        roots = torch.zeros((3, N, nb), dtype=torch.int32, device="cuda")
        msb = torch.zeros((3, N, s), dtype=torch.uint8, device="cuda")
        ipc.ipc_compare([zc[j] for j in range(3)], [zm[j] for j in range(3)], ldz, N, s, 0, tags, w.prf_seeds,
                        w.thr_a, p, roots, nb, msb, s)
        bits = torch.zeros((3, Q), dtype=torch.uint8, device="cuda")
        ipc.ipc_or_finalize(roots, nb, nb, p, Q, R, tags, w.prf_seeds, bits)
        torch.cuda.synchronize()
        ipc.ipc_status()
        assert (msb.cpu().numpy() == small["ref"]["msb"]).all()
        assert (bits.cpu().numpy() == small["ref"]["bits"]).all()
    assert (oracle.reconstruct_bits(small["ref"]["bits"]) == small["match"]).all()


def test_compare_multiblock_ragged_matches_oracle(torch):
    """The comparison kernel over several full OR blocks and a ragged last one. With
    1,024-row blocks, eight threads take four words each: the last block's parts hold
    4, 4, 4, 4, 4, 2 (the second ragged), 0 and 0 words. Block sizes of 8 and 2 words
    split down to single words. MSB shares are compared with the oracle at a row offset
    (global PRF counters), and opened-query bit shares with the oracle's OR tree from row 0."""
    ipc = lib()
    Q, R = 1, 31
    N, s = Q * R, 2 * 1024 + 21 * 32 + 9
    ldz = (s + 7) // 8 * 8
    rng = np.random.default_rng(2729)
    ml = rng.integers(0, 12801, size=(N, s))
    dot = rng.integers(-(ml // 8), ml // 8 + 1)  # hd / ml near 1/2: no match
    dot[7, 1100:1164] = ml[7, 1100:1164]  # identical codes: matches in one block of rotation 7

    def share(v):
        c0 = rng.integers(0, 65536, size=v.shape)
        c1 = rng.integers(0, 65536, size=v.shape)
        return np.stack([c0, c1, (v - c0 - c1) & 0xFFFF]).astype(np.uint16)

    zc_h, zm_h = share(dot), share(ml)
    zc = torch.zeros((3, N, ldz), dtype=torch.int16, device="cuda")
    zm = torch.zeros((3, N, ldz), dtype=torch.int16, device="cuda")
    zc[:, :, :s] = torch.from_numpy(zc_h.view(np.int16)).cuda()
    zm[:, :, :s] = torch.from_numpy(zm_h.view(np.int16)).cuda()
    seeds = (0x5EED0, 0x5EED1, 0x5EED2)
    tags = torch.from_numpy(tags_for(REQ, Q, R).view(np.int32)).cuda()
    cfg = oracle.mpc_cfg(seeds, req=REQ)

    def ref_msb(row0):
        out = np.zeros((3, N, s), np.uint8)
        for n in range(N):
            for i in range(s):
                out[:, n, i] = oracle.mpc_compare(cfg, zc_h[:, n, i], zm_h[:, n, i], 0, n, row0 + i)[0]
        return out

    for row0 in (65536, 0):
        want = ref_msb(row0)
        for p in (5, 3, 1):
            nb = (s + (32 << p) - 1) >> (5 + p)
            ld_roots = (row0 >> (5 + p)) + nb
            roots = torch.zeros((3, N, ld_roots), dtype=torch.int32, device="cuda")
            msb = torch.zeros((3, N, s), dtype=torch.uint8, device="cuda")
            ipc.ipc_compare([zc[j] for j in range(3)], [zm[j] for j in range(3)], ldz, N, s, row0, tags, seeds,
                            16384, p, roots, ld_roots, msb, s)
            torch.cuda.synchronize()
            ipc.ipc_status()
            assert (msb.cpu().numpy() == want).all(), (row0, p)
            if row0 == 0:
                bits = torch.zeros((3, Q), dtype=torch.uint8, device="cuda")
                ipc.ipc_or_finalize(roots, ld_roots, nb, p, Q, R, tags, seeds, bits)
                torch.cuda.synchronize()
                ipc.ipc_status()
                assert (bits.cpu().numpy()[:, 0] == oracle.or_tree(cfg, want, 0)).all(), p
                assert oracle.reconstruct_bits(bits.cpu().numpy())[0] == 1  # the planted matches
    # the opened MSBs are the plaintext rule: only the planted rows with ml > 0 match
    opened = want[0] ^ want[1] ^ want[2]
    assert opened.sum() == opened[7, 1100:1164].sum() == (ml[7, 1100:1164] > 0).sum()


@pytest.mark.parametrize("path", ["i8mma", "i8mix", "i32", "tc"])
def test_context_end_to_end_small(small, torch, path):
    ipc = lib()
    w = small["w"]
    ctx = make_ctx(w, path=path, keep=True, chunk_rows=1024 if path == "i8mma" else 0)
    try:
        load_workload(ctx, w, chunk=300)   # several loads, the middle ones ragged
        assert ipc.ipc_db_rows(ctx) == w.s
        qcode, qmask = query_shares_gpu(w, small["qc"], small["qm"])
        rid = ipc.submit_queries(ctx, [qcode[j] for j in range(3)], [qmask[j] for j in range(3)], w.Q, 1)
        sh = np.zeros((3, w.Q), np.uint8)
        ipc.fetch_bit_shares(ctx, rid, sh, w.Q, 60000)
        ref = oracle.mpc_match(oracle.mpc_cfg(w.prf_seeds, req=rid), oracle.iris_geom(), small["dbc"], small["dbm"],
                               small["qsc"], small["qsm"], want_z=True)
        assert (sh == ref["bits"]).all()
        # every A4 message and output component, through the transcript fingerprint
        assert ipc.fetch_transcript_hash(ctx, rid) == oracle.transcript_hash(ref["z_code"], ref["z_mask"], ref["bits"])
        for q, rho in ((0, 0), (1, 15), (4, 30)):
            dot = np.zeros(w.s, np.int16)
            ml = np.zeros(w.s, np.uint16)
            ipc.fetch_distances(ctx, rid, q, rho, 0, w.s, dot, ml)
            assert (ml == small["ml"][q, rho]).all()
            assert (dot == small["ml"][q, rho] - 2 * small["hd"][q, rho]).all()
        bits = np.zeros(w.Q, np.uint8)
        ipc.fetch_match_bits(ctx, rid, bits, w.Q, 60000)
        assert (bits == small["match"]).all()
        assert sorted(np.nonzero(bits)[0].tolist()) == w.planted_set().tolist()
    finally:
        ipc.ipc_destroy(ctx)


def test_context_multi_chunk(torch):
    """Three resident chunks (1024 rows each, the last ragged) and several loads."""
    ipc = lib()
    w = synth.Workload("chunks", s=2500, Q=3, rot_lo=-1, R=3, planted=1, seed=0xC0FFEE)
    dc, dm = w.db_bits()
    qc, qm = w.query_bits()
    dbc, dbm = oracle.encode_share(dc, dm, L, w.db_share_seed, 0)
    qsc, qsm = oracle.encode_share(qc, qm, L, w.q_share_seed, 1)
    match, _, _ = oracle.plain_match(oracle.Geom(16, 200, 4, -1, 3), qc, qm, dc, dm)
    for path in ("i8mma", "i8mix", "i32", "tc"):
        ctx = make_ctx(w, path=path, chunk_rows=1024)
        try:
            load_workload(ctx, w, chunk=700)
            qcode, qmask = query_shares_gpu(w, qc, qm)
            rid = ipc.submit_queries(ctx, [qcode[j] for j in range(3)], [qmask[j] for j in range(3)], w.Q, 1)
            sh = np.zeros((3, w.Q), np.uint8)
            ipc.fetch_bit_shares(ctx, rid, sh, w.Q, 60000)
            ref = oracle.mpc_match(oracle.mpc_cfg(w.prf_seeds, req=rid), oracle.Geom(16, 200, 4, -1, 3), dbc, dbm,
                                   qsc, qsm)
            assert (sh == ref["bits"]).all()
            assert (oracle.reconstruct_bits(sh) == match).all()
        finally:
            ipc.ipc_destroy(ctx)


def test_gemm_exact_at_max_length_and_extreme_limbs(torch):
    # l = 16384 (largest accepted, Lemma 2 with b = 2^16) and every element 0x7F80, whose limbs are
    # (-128, -128): the int32 partial sums reach 2^30 without wrapping; both paths must agree with
    # the exact ring product.
    ipc = lib()
    Lm = 16384
    s, Q, R = 130, 1, 3
    g = ipc.ipc_geom(16, 256, 4, -1, R)
    x = torch.full((s, Lm), 0x7F80, dtype=torch.int32).to(torch.int16).cuda()
    lo = torch.empty((s, Lm), dtype=torch.int8, device="cuda")
    hi = torch.empty((s, Lm), dtype=torch.int8, device="cuda")
    ipc.ipc_split_limbs(x, x.numel(), lo, hi)
    y = torch.full((3, Q, Lm), 0x7F80, dtype=torch.int32).to(torch.int16).cuda()
    y[2] = 0  # party 0's operand is [y_0 + y_2 | y_0] = [0x7F80 | 0x7F80]: C reaches 2l * 2 * 128^2 = 2^30
    tags = torch.from_numpy(tags_for(1, Q, R).view(np.int32)).cuda()
    res = {}
    for path in ("i8mma", "i8mix", "i32", "tc"):
        tc = path == "tc"
        blo = torch.empty((128, 2 * Lm), dtype=torch.int16 if tc else torch.int8, device="cuda")
        bhi = torch.empty((128, 2 * Lm), dtype=torch.int16 if tc else torch.int8, device="cuda")
        (ipc.ipc_prep_query_f16 if tc else ipc.ipc_prep_query)(y, Q, g, 0, blo, bhi, 128)
        z = torch.zeros((Q * R, 136), dtype=torch.int16, device="cuda")
        if tc:
            ipc.ipc_ring_gemm_tc([lo, lo], [hi, hi], s, blo, bhi, Q * R, 128, Lm, tags, 0, 0, 0, z, 136, 0)
        else:
            ipc.ipc_ring_gemm(path, [lo, lo], [hi, hi], s, blo, bhi, Q * R, 128, Lm, tags, 0, 0, 0, z, 136, 0)
        torch.cuda.synchronize()
        ipc.ipc_status()
        res[path] = u16(z)[:, :s]
    # equal seeds: the zero share is F - F = 0; z = sum over 2l of 0x7F80^2 (mod 2^16)
    expect = (2 * Lm * 0x7F80 * 0x7F80) & 0xFFFF
    for path in res:
        assert (res[path] == expect).all(), path


def test_degenerate_queries(torch):
    """All-masked query (ml = 0: never a match), a query equal to a database row (match at
    shift 0), a single-row database and a single rotation."""
    ipc = lib()
    w = synth.Workload("deg", s=1, Q=2, rot_lo=0, R=1, seed=77)
    dc, dm = w.db_bits()
    qc = np.stack([dc[0], dc[0]])
    qm = np.stack([np.zeros_like(dm[0]), dm[0]])
    ctx = make_ctx(w, path="i8mma")
    try:
        load_workload(ctx, w)
        qcode, qmask = query_shares_gpu(w, qc, qm)
        rid = ipc.submit_queries(ctx, [qcode[j] for j in range(3)], [qmask[j] for j in range(3)], 2, 1)
        bits = np.zeros(2, np.uint8)
        ipc.fetch_match_bits(ctx, rid, bits, 2, 60000)
        assert bits.tolist() == [0, 1]
    finally:
        ipc.ipc_destroy(ctx)


def test_empty_and_invalid_calls_are_rejected_without_launch(torch):
    ipc = lib()
    z = torch.zeros(8, dtype=torch.int16, device="cuda")
    with pytest.raises(ipc.IpcError):
        ipc.ipc_split_limbs(z, 0, z, z)
    w = synth.Workload("e", s=8, Q=1, R=1, rot_lo=0)
    ctx = make_ctx(w)
    try:
        code = torch.zeros((3, 1, L), dtype=torch.int16, device="cuda")
        with pytest.raises(ipc.IpcError):   # no database rows yet
            ipc.submit_queries(ctx, [code[j] for j in range(3)], [code[j] for j in range(3)], 1, 1)
        with pytest.raises(ipc.IpcError):   # more queries than configured
            ipc.submit_queries(ctx, [code[j] for j in range(3)], [code[j] for j in range(3)], 2, 1)
        with pytest.raises(ipc.IpcError):
            ipc.fetch_match_bits(ctx, 12345, np.zeros(1, np.uint8), 1, 0)
    finally:
        ipc.ipc_destroy(ctx)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_gemm_variants_and_tile_lists_match_int32(torch, variant):
    """Every GEMM variant (mixed / tensor-only with 128, 64, 32-column tiles), over all tiles and
    over a sparse list of column tiles, equals the int32 path on random full-range operands."""
    ipc = lib()
    rows, N, n_pad = 1000, 300, 384
    g = torch.Generator(device="cpu").manual_seed(variant)
    planes = [torch.randint(-128, 128, (rows, L), dtype=torch.int8, generator=g).cuda() for _ in range(4)]
    blo = torch.randint(-128, 128, (n_pad, 2 * L), dtype=torch.int8, generator=g).cuda()
    bhi = torch.randint(-128, 128, (n_pad, 2 * L), dtype=torch.int8, generator=g).cuda()
    tags = torch.from_numpy(tags_for(3, 10, 30).view(np.int32)).cuda()
    ldz = 1000
    ref = torch.zeros((N, ldz), dtype=torch.int16, device="cuda")
    ipc.ipc_ring_gemm("i32", planes[0:2], planes[2:4], rows, blo, bhi, N, n_pad, L, tags, 5, 6, 1, ref, ldz, 8)
    z = torch.zeros((N, ldz), dtype=torch.int16, device="cuda")
    ipc.ipc_ring_gemm_tiles(variant, planes[0:2], planes[2:4], rows, blo, bhi, N, n_pad, L, tags, 5, 6, 1, z, ldz, 8)
    torch.cuda.synchronize()
    ipc.ipc_status()
    assert (z.cpu() == ref.cpu()).all()
    bq = (128, 128, 64, 32)[variant]
    ntile = (N + bq - 1) // bq
    chosen = [t for t in range(ntile) if t % 3 != 1]
    lst = torch.tensor(chosen, dtype=torch.int32, device="cuda")
    cnt = torch.tensor([len(chosen)], dtype=torch.int32, device="cuda")
    z2 = torch.full((N, ldz), 77, dtype=torch.int16, device="cuda")
    ipc.ipc_ring_gemm_tiles(variant, planes[0:2], planes[2:4], rows, blo, bhi, N, n_pad, L, tags, 5, 6, 1, z2, ldz, 8,
                            lst, cnt)
    torch.cuda.synchronize()
    ipc.ipc_status()
    z2, refc = z2.cpu(), ref.cpu()
    for t in range(ntile):
        cols = slice(t * bq, min(N, (t + 1) * bq))
        if t in chosen:
            assert (z2[cols, :rows] == refc[cols, :rows]).all(), t
        else:
            assert (z2[cols] == 77).all(), t


def _f16(torch, t):
    """int8 limb tensor -> the fp16 bit patterns of the same integers (test-side conversion of the
    query operand)."""
    return t.to(torch.float16).view(torch.int16).contiguous()


@pytest.mark.parametrize("rows,N,row0", [(1000, 300, 8), (128, 256, 0), (4097, 31, 65536)])
def test_tc_gemm_matches_int32_on_random_limbs(torch, rows, N, row0):
    """The tcgen05 path equals the int32 path on random full-range limbs: ragged row tiles, one
    and two 256-column tiles (the second ragged), a row offset inside and past the first chunk."""
    ipc = lib()
    n_pad = (N + 127) // 128 * 128
    g = torch.Generator(device="cpu").manual_seed(rows + N)
    planes = [torch.randint(-128, 128, (rows, L), dtype=torch.int8, generator=g).cuda() for _ in range(4)]
    blo = torch.randint(-128, 128, (n_pad, 2 * L), dtype=torch.int8, generator=g).cuda()
    bhi = torch.randint(-128, 128, (n_pad, 2 * L), dtype=torch.int8, generator=g).cuda()
    tags = torch.from_numpy(tags_for(3, (N + 30) // 31, 31).view(np.int32)).cuda()
    ldz = (rows + 7) // 8 * 8
    ref = torch.zeros((N, ldz), dtype=torch.int16, device="cuda")
    ipc.ipc_ring_gemm("i32", planes[0:2], planes[2:4], rows, blo, bhi, N, n_pad, L, tags, 5, 6, 1, ref, ldz, row0)
    z = torch.full((N, ldz), 77, dtype=torch.int16, device="cuda")
    ipc.ipc_ring_gemm_tc(planes[0:2], planes[2:4], rows, _f16(torch, blo), _f16(torch, bhi), N, n_pad, L, tags, 5, 6,
                         1, z, ldz, row0)
    torch.cuda.synchronize()
    ipc.ipc_status()
    assert (z.cpu()[:, :rows] == ref.cpu()[:, :rows]).all()
    assert (z.cpu()[:, rows:] == 77).all()


@pytest.mark.parametrize("tile_cols", [256, 128])
def test_tc_tile_lists_match_int32(torch, tile_cols):
    """tcgen05 path with 256- and 128-column tiles: all tiles, then a sparse device-side list of
    column tiles walked by persistent CTAs (unlisted columns untouched)."""
    ipc = lib()
    rows, N, n_pad = 1000, 700, 768
    g = torch.Generator(device="cpu").manual_seed(tile_cols)
    planes = [torch.randint(-128, 128, (rows, L), dtype=torch.int8, generator=g).cuda() for _ in range(4)]
    blo = torch.randint(-128, 128, (n_pad, 2 * L), dtype=torch.int8, generator=g).cuda()
    bhi = torch.randint(-128, 128, (n_pad, 2 * L), dtype=torch.int8, generator=g).cuda()
    tags = torch.from_numpy(tags_for(4, 23, 31).view(np.int32)).cuda()
    ldz = 1000
    ref = torch.zeros((N, ldz), dtype=torch.int16, device="cuda")
    ipc.ipc_ring_gemm("i32", planes[0:2], planes[2:4], rows, blo, bhi, N, n_pad, L, tags, 5, 6, 0, ref, ldz, 16)
    p16 = planes
    b16 = [_f16(torch, blo), _f16(torch, bhi)]
    z = torch.zeros((N, ldz), dtype=torch.int16, device="cuda")
    ipc.ipc_ring_gemm_tc_tiles(tile_cols, p16[0:2], p16[2:4], rows, b16[0], b16[1], N, n_pad, L, tags, 5, 6, 0, z,
                               ldz, 16)
    torch.cuda.synchronize()
    ipc.ipc_status()
    refc = ref.cpu()
    assert (z.cpu()[:, :rows] == refc[:, :rows]).all()
    ntile = (N + tile_cols - 1) // tile_cols
    chosen = [t for t in range(ntile) if t != 1] if ntile > 2 else [ntile - 1]
    lst = torch.tensor(chosen, dtype=torch.int32, device="cuda")
    cnt = torch.tensor([len(chosen)], dtype=torch.int32, device="cuda")
    z2 = torch.full((N, ldz), 77, dtype=torch.int16, device="cuda")
    ipc.ipc_ring_gemm_tc_tiles(tile_cols, p16[0:2], p16[2:4], rows, b16[0], b16[1], N, n_pad, L, tags, 5, 6, 0, z2,
                               ldz, 16, lst, cnt)
    torch.cuda.synchronize()
    ipc.ipc_status()
    z2 = z2.cpu()
    for t in range(ntile):
        cols = slice(t * tile_cols, min(N, (t + 1) * tile_cols))
        if t in chosen:
            assert (z2[cols, :rows] == refc[cols, :rows]).all(), t
        else:
            assert (z2[cols] == 77).all(), t
    # an empty list launches nothing that writes
    cnt0 = torch.zeros(1, dtype=torch.int32, device="cuda")
    z3 = torch.full((N, ldz), 77, dtype=torch.int16, device="cuda")
    ipc.ipc_ring_gemm_tc_tiles(tile_cols, p16[0:2], p16[2:4], rows, b16[0], b16[1], N, n_pad, L, tags, 5, 6, 0, z3,
                               ldz, 16, lst, cnt0)
    torch.cuda.synchronize()
    assert (z3.cpu() == 77).all()


# ---------------------------------------------------------------------------------------------
# Galois-ring Shamir dot products (Sec. 4.3.2): IPC_PATH_TCG
# ---------------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small_galois(small):
    w = small["w"]
    dbc, dbm = oracle.encode_share_galois(small["dc"], small["dm"], L, w.db_share_seed, 0)
    qsc, qsm = oracle.encode_share_galois(small["qc"], small["qm"], L, w.q_share_seed, 1)
    ref = oracle.mpc_match_galois(oracle.mpc_cfg(w.prf_seeds, req=REQ), oracle.iris_geom(), dbc, dbm, qsc, qsm,
                                  want_z=True)
    return dict(dbc=dbc, dbm=dbm, qsc=qsc, qsm=qsm, ref=ref)


def test_encode_share_galois_matches_oracle(small, small_galois):
    w = small["w"]
    code, mask = encode_gpu(small["dc"], small["dm"], L, w.db_share_seed, 0, galois_shares=True)
    assert (u16(code) == small_galois["dbc"]).all()
    assert (u16(mask) == small_galois["dbm"]).all()
    qcode, qmask = encode_gpu(small["qc"], small["qm"], L, w.q_share_seed, 1, galois_shares=True)
    assert (u16(qcode) == small_galois["qsc"]).all() and (u16(qmask) == small_galois["qsm"]).all()


def test_prep_query_galois_is_lambda_times_rotated_share(small, small_galois, torch):
    """B_p = lambda_p * (rotated party-p share), elementwise in GR; multiplication by a0 + a1 X
    taken as the matrix a0 I + a1 [[0, 1], [1, 1]] on the coefficient pair."""
    ipc = lib()
    g = ipc.iris_geom()
    og = oracle.iris_geom()
    Q, R = 5, 31
    lam = oracle.gr_lagrange().astype(np.int64)
    y = torch.from_numpy(small_galois["qsc"].view(np.int16).copy()).cuda()
    n_pad = 256
    for party in range(3):
        lo = torch.empty((n_pad, L), dtype=torch.int16, device="cuda")
        hi = torch.empty((n_pad, L), dtype=torch.int16, device="cuda")
        ipc.ipc_prep_query_galois(y, Q, g, party, lo, hi, n_pad)
        lof = lo.view(torch.float16).float().cpu().numpy().astype(np.int64)
        hif = hi.view(torch.float16).float().cpu().numpy().astype(np.int64)
        rebuilt = (256 * hif + lof) & 0xFFFF
        l0, l1 = lam[party]
        for q in (0, 4):
            for rho in (0, 15, 30):
                v = oracle.rotate_u16(og, small_galois["qsc"][party, q], -15 + rho).astype(np.int64)
                y0, y1 = v[0::2], v[1::2]
                expect = np.empty(L, np.int64)
                expect[0::2] = (l0 * y0 + l1 * y1) & 0xFFFF
                expect[1::2] = (l0 * y1 + l1 * (y0 + y1)) & 0xFFFF
                assert (rebuilt[q * R + rho] == expect).all(), (party, q, rho)
        assert (rebuilt[Q * R:] == 0).all()


def test_ring_gemm_galois_matches_oracle_shares(small, small_galois, torch):
    ipc = lib()
    g = ipc.iris_geom()
    w = small["w"]
    Q, R, s = w.Q, w.R, w.s
    N, n_pad, ldz = Q * R, 256, 784
    tags = torch.from_numpy(tags_for(REQ, Q, R).view(np.int32)).cuda()
    for vec, (db, qs, key) in enumerate(((small_galois["dbc"], small_galois["qsc"], "z_code"),
                                         (small_galois["dbm"], small_galois["qsm"], "z_mask"))):
        planes = _planes(torch, db)
        y = torch.from_numpy(qs.view(np.int16).copy()).cuda()
        z = torch.zeros((3, N, ldz), dtype=torch.int16, device="cuda")
        for i in range(3):
            prev = (i + 2) % 3
            blo = torch.empty((n_pad, L), dtype=torch.int16, device="cuda")
            bhi = torch.empty((n_pad, L), dtype=torch.int16, device="cuda")
            ipc.ipc_prep_query_galois(y, Q, g, i, blo, bhi, n_pad)
            ipc.ipc_ring_gemm_tc_galois(256, planes[i][0], planes[i][1], s, blo, bhi, N, n_pad, L, tags,
                                        w.prf_seeds[i], w.prf_seeds[prev], vec, z[i], ldz, 0)
        torch.cuda.synchronize()
        ipc.ipc_status()
        assert (u16(z)[:, :, :s] == small_galois["ref"][key]).all(), key
    n = Q * R
    assert (oracle.reconstruct_u16(small_galois["ref"]["z_mask"]) == small["ml"].reshape(n, -1)).all()


@pytest.mark.parametrize("chunk_rows", [0, 1024])
def test_context_galois_end_to_end(small, small_galois, torch, chunk_rows):
    ipc = lib()
    w = small["w"]
    ctx = make_ctx(w, path="tcg", keep=True, chunk_rows=chunk_rows)
    try:
        load_workload(ctx, w, chunk=300, galois_shares=True)
        qcode, qmask = query_shares_gpu(w, small["qc"], small["qm"], galois_shares=True)
        rid = ipc.submit_queries(ctx, [qcode[j] for j in range(3)], [qmask[j] for j in range(3)], w.Q, 1)
        sh = np.zeros((3, w.Q), np.uint8)
        ipc.fetch_bit_shares(ctx, rid, sh, w.Q, 60000)
        ref = oracle.mpc_match_galois(oracle.mpc_cfg(w.prf_seeds, req=rid), oracle.iris_geom(), small_galois["dbc"],
                                      small_galois["dbm"], small_galois["qsc"], small_galois["qsm"], want_z=True)
        assert (sh == ref["bits"]).all()
        assert ipc.fetch_transcript_hash(ctx, rid) == oracle.transcript_hash(ref["z_code"], ref["z_mask"], ref["bits"])
        for q, rho in ((0, 0), (1, 15), (4, 30)):
            dot = np.zeros(w.s, np.int16)
            ml = np.zeros(w.s, np.uint16)
            ipc.fetch_distances(ctx, rid, q, rho, 0, w.s, dot, ml)
            assert (ml == small["ml"][q, rho]).all()
            assert (dot == small["ml"][q, rho] - 2 * small["hd"][q, rho]).all()
        bits = np.zeros(w.Q, np.uint8)
        ipc.fetch_match_bits(ctx, rid, bits, w.Q, 60000)
        assert (bits == small["match"]).all()
    finally:
        ipc.ipc_destroy(ctx)
