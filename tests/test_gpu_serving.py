"""Serving (continuous batching): every request's result is the oracle's, alone and in the mix.

A 2,200-row database in three resident chunks of 1,024 rows (the last ragged), 3 rotations,
six requests of 1-4 queries. The pool holds 6 query slots (fewer than the 15 queries
submitted), so later requests are admitted only as earlier ones finish, and they start at
whatever chunk the loop is on. Each request's three bit components must equal the 3-party
oracle's for its own request id, and its opened bits the plaintext matcher's, whatever else
ran beside it; the same request served alone gives the same opened bits.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_common import galois, lib, load_workload, make_ctx

pytestmark = pytest.mark.gpu

L = 12800
BATCHES = [(0, 3), (3, 2), (5, 1), (6, 4), (10, 2), (12, 3)]  # (first query, queries)


@pytest.fixture(scope="module")
def wl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = synth.Workload("serve", s=2200, Q=15, rot_lo=-1, R=3, planted=3, seed=0x5E77E)
    dc, dm = w.db_bits()
    qc, qm = w.query_bits()
    g = oracle.Geom(16, 200, 4, -1, 3)
    dbc, dbm = oracle.encode_share(dc, dm, L, w.db_share_seed, 0)
    qsc, qsm = oracle.encode_share(qc, qm, L, w.q_share_seed, 1)
    match, _, _ = oracle.plain_match(g, qc, qm, dc, dm, threads=os.cpu_count() or 1)
    gdbc, gdbm = oracle.encode_share_galois(dc, dm, L, w.db_share_seed, 0)
    gqsc, gqsm = oracle.encode_share_galois(qc, qm, L, w.q_share_seed, 1)
    return dict(w=w, g=g, dbc=dbc, dbm=dbm, qsc=qsc, qsm=qsm, match=match, ref={},
                galois=dict(dbc=gdbc, dbm=gdbm, qsc=gqsc, qsm=gqsm))


def _shares(wl, path):
    return wl["galois"] if galois(path) else wl


def _oracle_bits(wl, rid, q0, n, path="tc"):
    key = (rid, q0, n, galois(path))
    if key not in wl["ref"]:
        w = wl["w"]
        sh = _shares(wl, path)
        fn = oracle.mpc_match_galois if galois(path) else oracle.mpc_match
        ref = fn(oracle.mpc_cfg(w.prf_seeds, req=rid), wl["g"], sh["dbc"], sh["dbm"], sh["qsc"][:, q0:q0 + n],
                 sh["qsm"][:, q0:q0 + n])
        wl["ref"][key] = ref["bits"]
    return wl["ref"][key]


def _serve(wl, path, variant, pool, batches, tune_cache=None):
    ipc = lib()
    w = wl["w"]
    ctx = make_ctx(w, path=path, chunk_rows=1024, max_queries=4)
    sh = _shares(wl, path)
    try:
        load_workload(ctx, w, chunk=700, galois_shares=galois(path))
        ipc.ipc_serve_start(ctx, pool_queries=pool, variant=variant, tune_cache=tune_cache)
        tuning = ipc.ipc_serve_tuning(ctx)
        rids = []
        for q0, n in batches:
            code = [np.ascontiguousarray(sh["qsc"][j, q0:q0 + n]) for j in range(3)]
            mask = [np.ascontiguousarray(sh["qsm"][j, q0:q0 + n]) for j in range(3)]
            rids.append(ipc.ipc_serve_submit(ctx, code, mask, n))
        out = []
        for rid, (q0, n) in zip(rids, batches):
            got = np.zeros((3, n), np.uint8)
            ipc.fetch_bit_shares(ctx, rid, got, n, 120000)
            out.append((rid, q0, n, got, ipc.ipc_serve_times(ctx, rid)))
        stats = ipc.ipc_serve_stats(ctx)
        for rid, _, n, _, _ in out:
            bits = np.zeros(n, np.uint8)
            ipc.fetch_match_bits(ctx, rid, bits, n, 0)   # opens and releases
        ipc.ipc_serve_stop(ctx)
    finally:
        ipc.ipc_destroy(ctx)
    return out, stats, tuning


def _check(wl, out, path="tc"):
    for rid, q0, n, sh, _ in out:
        assert (sh == _oracle_bits(wl, rid, q0, n, path)).all(), (rid, q0, n)
        assert (oracle.reconstruct_bits(sh) == wl["match"][q0:q0 + n]).all(), (rid, q0, n)


@pytest.mark.parametrize("variant", ["tc256", "tc128"])
def test_mix_equals_oracle_and_alone(wl, variant):
    out, stats, _ = _serve(wl, "tc", variant, 6, BATCHES)
    _check(wl, out)
    w = wl["w"]
    assert stats["completed"] == len(BATCHES)
    assert stats["comparisons"] == sum(n for _, n in BATCHES) * w.R * w.s
    assert stats["n_chunks"] == 3
    times = [t for *_, t in out]
    # continuous batching: some request was admitted while another was still running, and some
    # waited for slots that a finished request gave back
    assert any(a[1] < b[2] and b[1] < a[2] for i, a in enumerate(times) for b in times[i + 1:])
    assert any(b[1] >= a[2] for a in times for b in times if b is not a)
    # each request alone in a fresh loop: same opened bits, shares of its own request id
    for q0, n in (BATCHES[3], BATCHES[2]):
        alone, _, _ = _serve(wl, "tc", variant, 6, [(q0, n)])
        _check(wl, alone)
        mixed = next(o for o in out if o[1] == q0)
        assert (oracle.reconstruct_bits(alone[0][3]) == oracle.reconstruct_bits(mixed[3])).all()


def test_autotune_table_is_cached_and_reused(wl, tmp_path):
    cache = str(tmp_path / "tune.json")
    out, stats, tuning = _serve(wl, "tc", -1, 6, BATCHES[:3], tune_cache=cache)
    _check(wl, out)
    assert os.path.exists(cache) and '"buckets"' in tuning
    assert open(cache).read().strip() == tuning.strip()
    out2, _, tuning2 = _serve(wl, "tc", -1, 6, BATCHES[:3], tune_cache=cache)
    _check(wl, out2)
    assert tuning2.strip() == tuning.strip()   # read back, not measured again
    assert sum(stats["variant_steps"]) == stats["steps"]


def test_galois_path_serving(wl):
    """Galois-ring Shamir dot products in the serving loop: shares equal to the oracle's."""
    out, stats, _ = _serve(wl, "tcg", "tc256", 6, BATCHES)
    _check(wl, out, "tcg")
    assert stats["completed"] == len(BATCHES)


def test_int8_path_serving(wl):
    out, stats, _ = _serve(wl, "i8mix", "mix128", 6, BATCHES)
    _check(wl, out)
    assert stats["completed"] == len(BATCHES)


def test_serving_refuses_other_calls_and_bad_sizes(wl):
    ipc = lib()
    w = wl["w"]
    ctx = make_ctx(w, path="tc", chunk_rows=1024, max_queries=4)
    try:
        load_workload(ctx, w, chunk=1100)
        ipc.ipc_serve_start(ctx, pool_queries=6, variant="tc256")
        code = [np.ascontiguousarray(wl["qsc"][j, :5]) for j in range(3)]
        with pytest.raises(ipc.IpcError):   # more than max_queries
            ipc.ipc_serve_submit(ctx, code, code, 5)
        with pytest.raises(ipc.IpcError):   # the context serves; no stand-alone submissions
            ipc.submit_queries(ctx, code, code, 1, 0)
        with pytest.raises(ipc.IpcError):   # nor more rows
            ipc.load_db_shares(ctx, code, code, 1, 0)
        ipc.ipc_serve_stop(ctx)
        with pytest.raises(ipc.IpcError):
            ipc.ipc_serve_submit(ctx, code, code, 1)
    finally:
        ipc.ipc_destroy(ctx)
