"""Both eyes and inner-batch matching on the GPU (ipc_check_persons) against the oracle.

Two eye databases of 1,500 rows; six persons whose codes include a near-duplicate of a
database row (eye 0), a near-duplicate of an earlier person of the batch (eye 1), and an
exact repeat of an earlier person (eye 0). Every part's bit components must equal the
oracle's for its own request id, and the combined components too; the opened bits must be
the plaintext rule (any eye against its database, or against an earlier person)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import galois, lib, load_workload, make_ctx

pytestmark = pytest.mark.gpu

L = 12800
R, ROT_LO = 3, -1


def _flip(rng, row, frac=0.10):
    x = row.copy()
    for b in rng.choice(L, int(frac * L), replace=False):
        x[b // 64] ^= np.uint64(1) << np.uint64(b % 64)
    return x


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(0x9E75)
    dbs = [synth.Workload(f"eye{e}", s=1500, Q=1, rot_lo=ROT_LO, R=R, seed=0xE1E0 + e) for e in range(2)]
    dbits = [w.db_bits() for w in dbs]
    P = 6
    qc = [rng.integers(0, 2**63, size=(P, L // 64), dtype=np.int64).view(np.uint64).copy() for _ in range(2)]
    qm = [np.array([dbits[e][1][rng.integers(0, 1500)] for _ in range(P)]) for e in range(2)]
    qc[0][1] = _flip(rng, dbits[0][0][17])          # person 1, eye 0: near-duplicate of DB row 17
    qm[0][1] = dbits[0][1][17]
    qc[1][4] = _flip(rng, qc[1][2])                 # person 4, eye 1: near-duplicate of person 2
    qm[1][4] = qm[1][2]
    qc[0][5], qm[0][5] = qc[0][3].copy(), qm[0][3].copy()   # person 5 repeats person 3 (eye 0)
    g = oracle.Geom(16, 200, 4, ROT_LO, R)
    expect = np.zeros(P, np.uint8)
    for e in range(2):
        m_db, _, _ = oracle.plain_match(g, qc[e], qm[e], dbits[e][0], dbits[e][1])
        expect |= m_db
        for p in range(1, P):
            m_b, _, _ = oracle.plain_match(g, qc[e][p:p + 1], qm[e][p:p + 1], qc[e][:p], qm[e][:p])
            expect[p] |= m_b[0]
    assert expect.tolist() == [0, 1, 0, 0, 1, 1]
    return dict(dbs=dbs, dbits=dbits, qc=qc, qm=qm, g=g, P=P, expect=expect)


@pytest.mark.parametrize("path", ["tc", "tcg", "i8mix"])
def test_persons_match_oracle(setup, path):
    ipc = lib()
    P, g = setup["P"], setup["g"]
    gal = galois(path)
    enc = oracle.encode_share_galois if gal else oracle.encode_share
    seeds = setup["dbs"][0].prf_seeds
    ctxs = []
    try:
        for e in range(2):
            w = setup["dbs"][e]
            w.prf_seeds = seeds
            ctx = make_ctx(w, path=path, max_queries=P)
            load_workload(ctx, w, chunk=600, galois_shares=gal)
            ctxs.append(ctx)
        q_sh = [enc(setup["qc"][e], setup["qm"][e], L, 0x0E5EED, 1) for e in range(2)]
        code = [np.ascontiguousarray(q_sh[e][0][j]) for e in range(2) for j in range(3)]
        mask = [np.ascontiguousarray(q_sh[e][1][j]) for e in range(2) for j in range(3)]
        shares, ids = ipc.ipc_check_persons(ctxs, code, mask, P, 0, 120000)
    finally:
        for c in ctxs:
            ipc.ipc_destroy(c)
    assert (oracle.reconstruct_bits(shares) == setup["expect"]).all()
    # every part from the oracle with its own request id
    match_fn = oracle.mpc_match_galois if gal else oracle.mpc_match
    parts = []
    for e in range(2):
        w = setup["dbs"][e]
        dbc, dbm = enc(setup["dbits"][e][0], setup["dbits"][e][1], L, w.db_share_seed, 0)
        parts.append(match_fn(oracle.mpc_cfg(seeds, req=ids[e]), g, dbc, dbm, q_sh[e][0], q_sh[e][1])["bits"])
    for e in range(2):
        parts.append(oracle.mpc_match_batch(oracle.mpc_cfg(seeds, req=ids[2 + e]), g, q_sh[e][0], q_sh[e][1],
                                            galois=gal))
    combined = oracle.or_combine(oracle.mpc_cfg(seeds, req=ids[4]), np.stack(parts))
    assert (shares == combined).all()
    assert len(set(ids)) == 5
