"""GPU parity of the fused chunk step (ipc_config.fused): the six ring GEMMs of a chunk and the
comparison phase of each tile in one launch, then the block join of the part roots. Shares,
messages (transcript fingerprint) and opened bits are compared with the oracle's 3-party
simulation, and with the unfused context on the same inputs, on both sharings of the dots
(replicated, tc; Galois-ring Shamir, tcg)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import lib, load_workload, make_ctx, query_shares_gpu, torch_mod

pytestmark = pytest.mark.gpu

L = 12800


@pytest.fixture(scope="module")
def torch():
    t = torch_mod()
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def oracle_shares(w, path, rid, dc, dm, qc, qm, want_z=False):
    geom = oracle.Geom(w.rows, w.cols, w.cell, w.rot_lo, w.R)
    cfg = oracle.mpc_cfg(w.prf_seeds, req=rid)
    if path == "tcg":
        dbc, dbm = oracle.encode_share_galois(dc, dm, L, w.db_share_seed, 0)
        qsc, qsm = oracle.encode_share_galois(qc, qm, L, w.q_share_seed, 1)
        return oracle.mpc_match_galois(cfg, geom, dbc, dbm, qsc, qsm, want_z=want_z)
    dbc, dbm = oracle.encode_share(dc, dm, L, w.db_share_seed, 0)
    qsc, qsm = oracle.encode_share(qc, qm, L, w.q_share_seed, 1)
    return oracle.mpc_match(cfg, geom, dbc, dbm, qsc, qsm, want_z=want_z)


def run_ctx(w, path, fused, qc, qm, chunk_rows=0, keep=False, requests=1):
    """Loads w's database and submits the queries `requests` times; returns the contexts' (request
    id, bit shares, opened bits, transcript hash or None) per request."""
    ipc = lib()
    ctx = make_ctx(w, path=path, keep=keep, chunk_rows=chunk_rows, fused=fused, max_requests=max(2, requests))
    out = []
    try:
        load_workload(ctx, w, chunk=4096, galois_shares=path == "tcg")
        qcode, qmask = query_shares_gpu(w, qc, qm, galois_shares=path == "tcg")
        rids = [ipc.submit_queries(ctx, [qcode[j] for j in range(3)], [qmask[j] for j in range(3)], w.Q, 1)
                for _ in range(requests)]
        for rid in rids:
            sh = np.zeros((3, w.Q), np.uint8)
            ipc.fetch_bit_shares(ctx, rid, sh, w.Q, 120000)
            th = ipc.fetch_transcript_hash(ctx, rid) if keep else None
            bits = np.zeros(w.Q, np.uint8)
            ipc.fetch_match_bits(ctx, rid, bits, w.Q, 120000)
            out.append((rid, sh, bits, th))
    finally:
        ipc.ipc_destroy(ctx)
    return out


@pytest.mark.parametrize("path", ["tc", "tcg"])
def test_fused_matches_oracle_two_column_tiles(torch, path):
    """300 rows (three 128-row tiles, the last ragged; one ragged 1,024-row block), 9 queries x 31
    rotations = 279 columns (two 256-column tiles, the second with 23 columns), planted
    near-duplicates; every message through the transcript fingerprint."""
    w = synth.Workload("fused2", s=300, Q=9, planted=3, seed=0xF05ED)
    dc, dm = w.db_bits()
    qc, qm = w.query_bits()
    ((rid, sh, bits, th),) = run_ctx(w, path, True, qc, qm, keep=True)
    ref = oracle_shares(w, path, rid, dc, dm, qc, qm, want_z=True)
    assert (sh == ref["bits"]).all()
    assert th == oracle.transcript_hash(ref["z_code"], ref["z_mask"], ref["bits"])
    match, _, _ = oracle.plain_match(oracle.Geom(w.rows, w.cols, w.cell, w.rot_lo, w.R), qc, qm, dc, dm)
    assert (bits == match).all() and bits.sum() == len(w.planted_set())


@pytest.mark.parametrize("path", ["tc", "tcg"])
def test_fused_multi_chunk_and_requests_equal_unfused(torch, path):
    """Three 1,024-row chunks (the last ragged: 452 rows), 3 queries x 3 rotations, two requests in
    flight: shares equal to the oracle's and to the unfused context's for the same request ids."""
    w = synth.Workload("fusedc", s=2500, Q=3, rot_lo=-1, R=3, planted=1, seed=0xF05EE)
    dc, dm = w.db_bits()
    qc, qm = w.query_bits()
    fused = run_ctx(w, path, True, qc, qm, chunk_rows=1024, requests=2)
    plain = run_ctx(w, path, False, qc, qm, chunk_rows=1024, requests=2)
    for (rid, sh, bits, _), (rid2, sh2, bits2, _) in zip(fused, plain):
        assert rid == rid2
        assert (sh == sh2).all() and (bits == bits2).all()
        ref = oracle_shares(w, path, rid, dc, dm, qc, qm)
        assert (sh == ref["bits"]).all()
    match, _, _ = oracle.plain_match(oracle.Geom(w.rows, w.cols, w.cell, w.rot_lo, w.R), qc, qm, dc, dm)
    assert (fused[0][2] == match).all() and match.sum() == 1


@pytest.mark.parametrize("path", ["tc", "tcg"])
def test_fused_persistent_tiles(torch, path):
    """20,000 rows in one chunk: 157 row tiles, more than one per SM, so CTAs run several tiles of
    six passes back to back; 2 queries x 1 rotation. Shares equal to the oracle's."""
    w = synth.Workload("fusedp", s=20000, Q=2, rot_lo=0, R=1, planted=1, seed=0xF05EF)
    dc, dm = w.db_bits()
    qc, qm = w.query_bits()
    ((rid, sh, bits, _),) = run_ctx(w, path, True, qc, qm)
    ref = oracle_shares(w, path, rid, dc, dm, qc, qm)
    assert (sh == ref["bits"]).all()
    match, _, _ = oracle.plain_match(oracle.Geom(w.rows, w.cols, w.cell, w.rot_lo, w.R), qc, qm, dc, dm)
    assert (bits == match).all() and match.sum() == 1


@pytest.mark.parametrize("path", ["tc", "tcg"])
def test_fused_degenerate_queries(torch, path):
    """A one-row database (one row tile with one valid row: a part of one word of one row), one
    rotation, an all-masked query (ml = 0: never a match) and a query equal to the row (a match):
    shares equal to the oracle's, bits [0, 1]."""
    ipc = lib()
    w = synth.Workload("fusedd", s=1, Q=2, rot_lo=0, R=1, seed=78)
    dc, dm = w.db_bits()
    qc = np.stack([dc[0], dc[0]])
    qm = np.stack([np.zeros_like(dm[0]), dm[0]])
    ((rid, sh, bits, th),) = run_ctx(w, path, True, qc, qm, keep=True)
    ref = oracle_shares(w, path, rid, dc, dm, qc, qm, want_z=True)
    assert (sh == ref["bits"]).all()
    assert th == oracle.transcript_hash(ref["z_code"], ref["z_mask"], ref["bits"])
    assert bits.tolist() == [0, 1]


def test_fused_rejects_other_settings(torch):
    ipc = lib()
    w = synth.Workload("fusedx", s=300, Q=1, planted=0, seed=1)
    g = ipc.ipc_geom(w.rows, w.cols, w.cell, w.rot_lo, w.R)
    for kw in (dict(path="i8mma"), dict(path="tc", plain_mask=True), dict(path="tc", lift="const")):
        with pytest.raises(RuntimeError):
            ipc.ipc_create(ipc.make_config(g, fused=True, **kw))
