"""The lifting variants on the GPU (Sec. 5.1, Sec. 6.2 Table 2) against the oracle: ConstLift
(ml over Z_2^32) and NoLift (code and mask dot products over Z_2^32).

Stage by stage (A0 sharing, A1 limbs, A2 query operand, A3 ring GEMM over Z_2^32, the
lift-free comparison) and end to end through the context. Integers throughout: every
comparison is exact, shares included.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import encode_gpu32, lib, lift_shares, load_workload, make_ctx, tags_for, torch_mod

pytestmark = pytest.mark.gpu

L = 12800
REQ = 13


@pytest.fixture(scope="module")
def torch():
    t = torch_mod()
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def _from_limbs(torch, limbs):
    """Limb planes (int8, or int16 holding fp16 bit patterns) -> numpy uint32 values
    sum_i limb_i 2^(8i) mod 2^32."""
    acc = np.zeros(limbs[0].shape, np.int64)
    for i, t in enumerate(limbs):
        v = t.view(torch.float16).float() if t.dtype == torch.int16 else t
        acc += v.cpu().numpy().astype(np.int64) << (8 * i)
    return (acc & 0xFFFFFFFF).astype(np.uint32)


def test_split_limbs32_exact_on_edges_and_random(torch):
    ipc = lib()
    rng = np.random.default_rng(50)
    edges = [0, 1, 0x7F, 0x80, 0xFF, 0x100, 0x7FFF, 0x8000, 0xFFFF, 0x10000, 0x7F7F7F7F, 0x80808080, 0x7FFFFFFF,
             0x80000000, 0xFFFFFFFF, 0xFFFFFF80, 0x807F807F]
    x = np.concatenate([np.array(edges, np.uint32), rng.integers(0, 2**32, 1 << 20, dtype=np.uint64).astype(np.uint32),
                        np.arange(4096, dtype=np.uint32) * 0x00010001])
    n = x.size - 3   # a ragged tail for the 4-per-thread loop
    dx = torch.from_numpy(x.view(np.int32).copy()).cuda()
    limbs = [torch.full((x.size,), 77, dtype=torch.int8, device="cuda") for _ in range(4)]
    ipc.ipc_split_limbs32(dx, n, limbs)
    torch.cuda.synchronize()
    assert (_from_limbs(torch, [t[:n] for t in limbs]) == x[:n]).all()
    assert all((t.cpu()[n:] == 77).all() for t in limbs)


def test_encode_share32_matches_oracle(torch):
    w = synth.Workload("e32", s=300, Q=2, planted=1, seed=0xE32)
    dc, dm = w.db_bits()
    code, mask = encode_gpu32(dc, dm, L, w.db_share_seed, 0, idx0=5)
    rc, rm = oracle.encode_share32(dc, dm, L, w.db_share_seed, 0, idx0=5)
    assert (u32(code) == rc).all() and (u32(mask) == rm).all()


def test_prep_query32_is_rotated_aby3_operand(torch):
    ipc = lib()
    g, og = ipc.iris_geom(), oracle.iris_geom()
    Q, R, n_pad = 3, 31, 128
    rng = np.random.default_rng(51)
    y = rng.integers(0, 2**32, (3, Q, L), dtype=np.uint64).astype(np.uint32)
    dy = torch.from_numpy(y.view(np.int32).copy()).cuda()
    for party in range(3):
        prev = (party + 2) % 3
        for segments in (2, 1):
            b = [torch.empty((n_pad, segments * L), dtype=torch.int16, device="cuda") for _ in range(4)]
            ipc.ipc_prep_query32_f16(dy, Q, g, party, segments, b, n_pad)
            got = _from_limbs(torch, b)
            for q in (0, 2):
                for rho in (0, 15, 30):
                    rot = lambda v: (oracle.rotate_u16(og, (v & 0xFFFF).astype(np.uint16), rho - 15).astype(np.uint32)
                                     | (oracle.rotate_u16(og, (v >> 16).astype(np.uint16), rho - 15).astype(np.uint32)
                                        << 16))
                    own = rot(y[party, q])
                    if segments == 2:
                        both = rot((y[party, q].astype(np.uint64) + y[prev, q]).astype(np.uint32))
                        assert (got[q * R + rho, :L] == both).all()
                        assert (got[q * R + rho, L:] == own).all()
                    else:
                        assert (got[q * R + rho] == own).all()
            assert (got[Q * R:] == 0).all()


def _gemm_case(torch, rows, N, segments, row0, extreme=False, seeds=(5, 5), L=L):
    ipc = lib()
    n_pad = (N + 127) // 128 * 128
    K = segments * L
    g = torch.Generator(device="cpu").manual_seed(rows * 7 + N + segments)
    if extreme:   # every limb -128: each product 2^14, the accumulators at the edge of their window
        xl = [torch.full((rows, L), -128, dtype=torch.int8) for _ in range(4 * segments)]
        bl = [torch.full((n_pad, K), -128, dtype=torch.int8) for _ in range(4)]
    else:
        xl = [torch.randint(-128, 128, (rows, L), dtype=torch.int8, generator=g) for _ in range(4 * segments)]
        bl = [torch.randint(-128, 128, (n_pad, K), dtype=torch.int8, generator=g) for _ in range(4)]
    f16 = lambda t: t.to(torch.float16).view(torch.int16).contiguous().cuda()
    xd, bd = [t.contiguous().cuda() for t in xl], [f16(t) for t in bl]
    tags = torch.from_numpy(tags_for(3, (N + 30) // 31, 31)[:N].copy().view(np.int32)).cuda()
    ldz = (rows + 7) // 8 * 8
    z = torch.full((N, ldz), 77, dtype=torch.int32, device="cuda")
    ipc.ipc_ring_gemm_tc32(segments, xd, rows, bd, N, n_pad, L, tags, seeds[0], seeds[1], 1, z, ldz, row0)
    torch.cuda.synchronize()
    ipc.ipc_status()
    # exact reference: per limb pair (a, b) with a + b < 4 the integer product sum (below 2^29 in
    # magnitude, exact in fp64), then sum_s 2^(8s) S_s mod 2^32
    Xa = [torch.cat([xl[4 * s + a] for s in range(segments)], dim=1).double().cuda() for a in range(4)]
    Bb = [t[:N].double().cuda() for t in bl]
    ref = np.zeros((N, rows), np.int64)
    for a in range(4):
        for b in range(4 - a):
            S = (Bb[b] @ Xa[a].T).round().cpu().numpy().astype(np.int64)
            ref = (ref + ((S & 0xFFFFFFFF) << (8 * (a + b)))) & 0xFFFFFFFF
    return u32(z), ref.astype(np.uint32), tags


@pytest.mark.parametrize("rows,N,segments,row0", [(300, 200, 2, 0), (1000, 93, 2, 1024), (130, 128, 1, 0),
                                                    (260, 300, 2, 0)])
def test_gemm_tc32_exact_on_random_limbs(torch, rows, N, segments, row0):
    """Equal seeds make the zero share vanish: z is the exact ring product; ragged row and column
    tiles (one and two 256-column tiles), one and two K segments."""
    z, ref, _ = _gemm_case(torch, rows, N, segments, row0)
    assert (z[:, :rows] == ref).all()
    assert (z[:, rows:] == 77).all()


@pytest.mark.parametrize("l,segments", [(256, 1), (128, 2), (768, 1)])
def test_gemm_tc32_exact_at_short_k(torch, l, segments):
    """The shortest K, 256 (eight k-blocks: pass A four drain periods, pass B four stages with a
    single S_0 drain), over one segment and over two segments of 128 (the second segment
    starting at a pass-B stage), and K = 768 (three S_0 periods)."""
    z, ref, _ = _gemm_case(torch, 200, 280, segments, 0, L=l)
    assert (z[:, :200] == ref).all()
    ze, refe, _ = _gemm_case(torch, 128, 128, segments, 0, extreme=True, L=l)
    assert (ze[:, :128] == refe).all()


def test_gemm_tc32_exact_at_extreme_limbs(torch):
    z, ref, _ = _gemm_case(torch, 128, 128, 2, 0, extreme=True)
    assert (z[:, :128] == ref).all()


def test_gemm_tc32_zero_shares_match_oracle(torch):
    """Unequal seeds: z - (exact product) is F(seed_own) - F(seed_prev) of the D_ZA32 counters,
    checked through the oracle's dot on the same 32-bit vectors."""
    rows, N = 70, 31
    z, ref, _ = _gemm_case(torch, rows, N, 2, 2048, seeds=(11, 29))
    diff = (z[:, :rows].astype(np.int64) - ref.astype(np.int64)) & 0xFFFFFFFF
    cfg = oracle.mpc_cfg((11, 0, 29), req=3)
    zero = np.zeros((3, 1), np.uint32)
    for n in (0, 30):
        q, rho = n // 31, n % 31
        for r in (0, 1, 69):
            # party 0's component of a zero dot: F(seed_0) - F(seed_2) at global row 2048 + r
            z3 = oracle.mpc_dot32(cfg, zero, zero, q, rho, 2048 + r, 1)
            assert diff[n, r] == z3[0], (n, r)


def _cases(rng, n):
    out = []
    for ml in list(range(0, 40)) + [L] + [int(t) for t in rng.integers(0, L + 1, n)]:
        q4 = ml // 4
        for dot in (q4 - 1, q4, q4 + 1, -ml, ml, int(rng.integers(-ml, ml + 1))):
            if -ml <= dot <= ml:
                out.append((ml, dot))
    return out


@pytest.mark.parametrize("mode,thr_a,thr_b", [("const", 16384, 0), ("none", 16384, 0), ("none", 10000, 40000)])
def test_compare_liftfree_matches_oracle(torch, mode, thr_a, thr_b):
    ipc = lib()
    rng = np.random.default_rng(52)
    cases = _cases(rng, 150)[:992]
    n_cols, n_rows = 2, len(cases) // 2
    ldz = (n_rows + 7) // 8 * 8
    ml = np.zeros((n_cols, ldz), np.int64)
    dot = np.zeros((n_cols, ldz), np.int64)
    for k, (a, b) in enumerate(cases[:n_cols * n_rows]):
        ml[k // n_rows, k % n_rows], dot[k // n_rows, k % n_rows] = a, b
    wide = mode == "none"
    m = rng.integers(0, 2**32, (2, n_cols, ldz), dtype=np.uint64)
    ml_sh = np.stack([m[0], m[1], (ml.astype(np.uint64) - m[0] - m[1]) & np.uint64(0xFFFFFFFF)]).astype(np.uint32)
    mod = 2**32 if wide else 2**16
    d = rng.integers(0, mod, (2, n_cols, ldz), dtype=np.uint64)
    dsh = np.stack([d[0], d[1], (dot.astype(np.uint64) - d[0] - d[1]) & np.uint64(mod - 1)])
    dsh = dsh.astype(np.uint32 if wide else np.uint16)
    seeds = (0x71, 0x72, 0x73)
    tags = np.array([(REQ, 5), (REQ, (1 << 5) | 9)], np.uint32)
    dml = torch.from_numpy(ml_sh.view(np.int32).copy()).cuda()
    dd = torch.from_numpy(dsh.view(np.int32 if wide else np.int16).copy()).cuda()
    dtags = torch.from_numpy(tags.view(np.int32).copy()).cuda()
    nb = (n_rows + 1023) // 1024
    roots = torch.zeros((3, n_cols, nb), dtype=torch.int32, device="cuda")
    msb = torch.zeros((3, n_cols, n_rows), dtype=torch.uint8, device="cuda")
    dl = [dd[j] for j in range(3)]
    ipc.ipc_compare_liftfree(None if wide else dl, dl if wide else None, [dml[j] for j in range(3)], ldz, n_cols,
                             n_rows, 0, dtags, seeds, thr_a, thr_b, 5, roots, nb, msb, n_rows)
    torch.cuda.synchronize()
    ipc.ipc_status()
    got = msb.cpu().numpy()
    b = thr_b or 65536
    assert (oracle.reconstruct_bits(got) == (b * dot[:, :n_rows] > thr_a * ml[:, :n_rows])).all()
    cfg = oracle.mpc_cfg(seeds, req=REQ, thr_a=thr_a)
    omode = oracle.LIFT_NONE if wide else oracle.LIFT_CONST
    for c, (q, rho) in enumerate(((0, 5), (1, 9))):
        for r in range(0, n_rows, 3):
            ref, _ = oracle.mpc_compare_liftfree(cfg, omode, dsh[:, c, r], ml_sh[:, c, r], thr_b, q, rho, r)
            assert (got[:, c, r] == ref).all(), (c, r)


@pytest.fixture(scope="module")
def wl(torch):
    """1,500 rows in two 1,024-row chunks (the second ragged), 2 queries x 31 rotations."""
    w = synth.Workload("lift", s=1500, Q=2, planted=2, seed=0x11F8)
    dc, dm = w.db_bits()
    qc, qm = w.query_bits()
    match, ml, hd = oracle.plain_match(oracle.iris_geom(), qc, qm, dc, dm, distances=True)
    return dict(w=w, dc=dc, dm=dm, qc=qc, qm=qm, match=match, ml=ml, hd=hd)


@pytest.mark.parametrize("lift", ["const", "none"])
def test_context_lift_variant_matches_oracle(wl, torch, lift):
    ipc = lib()
    w = wl["w"]
    ctx = make_ctx(w, path="tc", keep=True, chunk_rows=1024, lift=lift)
    try:
        load_workload(ctx, w, chunk=700, lift=lift)
        assert ipc.ipc_db_rows(ctx) == w.s
        qcode, qmask = lift_shares(wl["qc"], wl["qm"], w.l, w.q_share_seed, 1, lift=lift)
        rid = ipc.submit_queries(ctx, [qcode[j] for j in range(3)], [qmask[j] for j in range(3)], w.Q, 1)
        sh = np.zeros((3, w.Q), np.uint8)
        ipc.fetch_bit_shares(ctx, rid, sh, w.Q, 60000)
        mode = oracle.LIFT_NONE if lift == "none" else oracle.LIFT_CONST
        c32, m32 = oracle.encode_share32(wl["dc"], wl["dm"], w.l, w.db_share_seed, 0)
        qc32, qm32 = oracle.encode_share32(wl["qc"], wl["qm"], w.l, w.q_share_seed, 1)
        if mode == oracle.LIFT_CONST:
            dbc = oracle.encode_share(wl["dc"], wl["dm"], w.l, w.db_share_seed, 0)[0]
            qsc = oracle.encode_share(wl["qc"], wl["qm"], w.l, w.q_share_seed, 1)[0]
        else:
            dbc, qsc = c32, qc32
        ref = oracle.mpc_match_lift(oracle.mpc_cfg(w.prf_seeds, req=rid), oracle.iris_geom(), mode, dbc, m32, qsc,
                                    qm32, want_z=True)
        assert (sh == ref["bits"]).all()
        assert ipc.fetch_transcript_hash(ctx, rid) == oracle.transcript_hash(ref["z_code"], ref["z_mask"], ref["bits"])
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


def test_lift_variant_refusals(wl, torch):
    ipc = lib()
    w = wl["w"]
    for kw in (dict(path="tcg", lift="const"), dict(path="i8mma", lift="none"),
               dict(path="tc", lift="const", thr_b=40000), dict(path="tc", lift="none", thr_b=70000)):
        with pytest.raises(ipc.IpcError):
            make_ctx(w, **kw)
    ctx = make_ctx(w, path="tc", chunk_rows=1024, lift="const")
    try:
        load_workload(ctx, w, chunk=1500, lift="const")
        with pytest.raises(ipc.IpcError):
            ipc.ipc_serve_start(ctx, pool_queries=4, variant="tc256")
    finally:
        ipc.ipc_destroy(ctx)
