"""Failure reporting without a GPU fault. A bounded wait that runs out (on a flag that nothing
sets) raises the device status word instead of trapping; the host reads it as IPC_EDEVICE, the
word is cleared, and a context keeps working afterwards."""
import time

import numpy as np
import pytest

import oracle
import synth
from gpu_common import lib, load_workload, make_ctx, query_shares_gpu, torch_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = torch_mod()
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def test_bounded_wait_reports_and_clears(torch):
    ipc = lib()
    ipc.ipc_status()                        # start clean
    t0 = time.perf_counter()
    ipc.ipc_selftest_bounded_wait(20000)    # gives up after 20 ms
    assert time.perf_counter() - t0 >= 0.02
    with pytest.raises(ipc.IpcError) as e:
        ipc.ipc_status()
    assert e.value.rc == ipc.IPC_EDEVICE
    ipc.ipc_status()                        # read once, then cleared
    with pytest.raises(ipc.IpcError):
        ipc.ipc_selftest_bounded_wait(0)


def test_context_reports_the_status_and_keeps_working(torch):
    ipc = lib()
    w = synth.Workload("fail", s=300, Q=2, planted=1, seed=0xFA11)
    ctx = make_ctx(w, path="tc")
    try:
        load_workload(ctx, w, chunk=300)
        qc, qm = w.query_bits()
        code, mask = query_shares_gpu(w, qc, qm)
        rid = ipc.submit_queries(ctx, [code[j] for j in range(3)], [mask[j] for j in range(3)], w.Q, 1)
        ipc.ipc_selftest_bounded_wait(1000)  # a wait on this device gives up while the request runs
        sh = np.zeros((3, w.Q), np.uint8)
        with pytest.raises(ipc.IpcError) as e:
            ipc.fetch_bit_shares(ctx, rid, sh, w.Q, 60000)
        assert e.value.rc == ipc.IPC_EDEVICE
        # the word is cleared and the request's results are intact
        ipc.fetch_bit_shares(ctx, rid, sh, w.Q, 60000)
        dc, dm = w.db_bits()
        dbc, dbm = oracle.encode_share(dc, dm, w.l, w.db_share_seed, 0)
        qsc, qsm = oracle.encode_share(qc, qm, w.l, w.q_share_seed, 1)
        ref = oracle.mpc_match(oracle.mpc_cfg(w.prf_seeds, req=rid), oracle.iris_geom(), dbc, dbm, qsc, qsm)
        assert (sh == ref["bits"]).all()
        ipc.ipc_release(ctx, rid)
        # and the context serves the next request normally
        rid2 = ipc.submit_queries(ctx, [code[j] for j in range(3)], [mask[j] for j in range(3)], w.Q, 1)
        bits = np.zeros(w.Q, np.uint8)
        ipc.fetch_match_bits(ctx, rid2, bits, w.Q, 60000)
        match, _, _ = oracle.plain_match(oracle.iris_geom(), qc, qm, dc, dm)
        assert (bits == match).all() and bits.sum() == w.planted
    finally:
        ipc.ipc_destroy(ctx)


# ---------------------------------------------------------------------------------------------
# Failure paths made on the host: nothing here faults, traps or hangs the GPU. Every wait that
# runs out is a bounded one (a device flag that nothing sets) or a host-side timeout.
# ---------------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small():
    w = synth.Workload("fail2", s=300, Q=2, planted=1, seed=0xFA12)
    qc, qm = w.query_bits()
    dc, dm = w.db_bits()
    dbc, dbm = oracle.encode_share(dc, dm, w.l, w.db_share_seed, 0)
    qsc, qsm = oracle.encode_share(qc, qm, w.l, w.q_share_seed, 1)
    match, _, _ = oracle.plain_match(oracle.iris_geom(), qc, qm, dc, dm)
    return dict(w=w, qc=qc, qm=qm, dbc=dbc, dbm=dbm, qsc=qsc, qsm=qsm, match=match)


def _oracle_shares(small, rid):
    w = small["w"]
    return oracle.mpc_match(oracle.mpc_cfg(w.prf_seeds, req=rid), oracle.iris_geom(), small["dbc"], small["dbm"],
                            small["qsc"], small["qsm"])["bits"]


def test_fetch_with_zero_timeout_on_a_running_request(torch, small):
    """fetch_match_bits with timeout 0 on a request that is still queued returns IPC_ETIMEOUT and
    keeps the request; a later fetch returns its bits. The request is held back by its inputs:
    they are produced on a stream that first spins for about 0.3 s (a kernel that ends by itself)."""
    ipc = lib()
    w = small["w"]
    ctx = make_ctx(w, path="tc")
    try:
        load_workload(ctx, w, chunk=300)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            torch.cuda._sleep(600_000_000)
            code, mask = query_shares_gpu(w, small["qc"], small["qm"])
        ipc.ipc_set_input_stream(ctx, side.cuda_stream)
        rid = ipc.submit_queries(ctx, [code[j] for j in range(3)], [mask[j] for j in range(3)], w.Q, 1)
        bits = np.zeros(w.Q, np.uint8)
        with pytest.raises(ipc.IpcError) as e:
            ipc.fetch_match_bits(ctx, rid, bits, w.Q, 0)
        assert e.value.rc == ipc.IPC_ETIMEOUT
        ipc.fetch_match_bits(ctx, rid, bits, w.Q, -1)
        assert (bits == small["match"]).all() and bits.sum() == w.planted
        side.synchronize()
    finally:
        ipc.ipc_destroy(ctx)


@pytest.mark.parametrize("fused", [False, True])
def test_dropped_party_times_out_instead_of_hanging(torch, small, fused):
    """A party that never delivers its messages (its stream waits for a flag that nothing sets,
    injected on the host): fetches with a shorter timeout return IPC_ETIMEOUT, the wait gives up
    after its limit and the request reports IPC_EDEVICE once; its results are intact and the next
    request is served normally. The same with the fused chunk step, whose launch waits for every
    party's query preparation."""
    ipc = lib()
    w = small["w"]
    ctx = make_ctx(w, path="tc", fused=fused)
    try:
        load_workload(ctx, w, chunk=300)
        code, mask = query_shares_gpu(w, small["qc"], small["qm"])
        # one ordinary request first: in a fresh process it also loads the library's kernels, which
        # would otherwise make the stalled request's submit outlast the stall
        bits = np.zeros(w.Q, np.uint8)
        ipc.fetch_match_bits(ctx, ipc.submit_queries(ctx, [code[j] for j in range(3)], [mask[j] for j in range(3)],
                                                     w.Q, 1), bits, w.Q, 60000)
        assert (bits == small["match"]).all()
        torch.cuda.synchronize()
        ipc.ipc_status()
        ipc.ipc_debug_stall_party(ctx, 1, 300000)   # party 1 is "gone" for 0.3 s
        t0 = time.perf_counter()
        rid = ipc.submit_queries(ctx, [code[j] for j in range(3)], [mask[j] for j in range(3)], w.Q, 1)
        sh = np.zeros((3, w.Q), np.uint8)
        with pytest.raises(ipc.IpcError) as e:
            ipc.fetch_bit_shares(ctx, rid, sh, w.Q, 50)
        assert e.value.rc == ipc.IPC_ETIMEOUT
        with pytest.raises(ipc.IpcError) as e:
            ipc.fetch_bit_shares(ctx, rid, sh, w.Q, -1)
        assert e.value.rc == ipc.IPC_EDEVICE
        assert time.perf_counter() - t0 >= 0.3
        ipc.fetch_bit_shares(ctx, rid, sh, w.Q, -1)
        assert (sh == _oracle_shares(small, rid)).all()
        ipc.ipc_release(ctx, rid)
        rid2 = ipc.submit_queries(ctx, [code[j] for j in range(3)], [mask[j] for j in range(3)], w.Q, 1)
        bits[:] = 0
        ipc.fetch_match_bits(ctx, rid2, bits, w.Q, 60000)
        assert (bits == small["match"]).all()
        with pytest.raises(ipc.IpcError):
            ipc.ipc_debug_stall_party(ctx, 3, 1000)
    finally:
        ipc.ipc_destroy(ctx)


def test_request_slots_exhausted_is_eagain(torch, small):
    """With two request slots, a third request submitted before any is fetched or released is
    refused with IPC_EAGAIN (nothing is allocated per request); releasing one makes room."""
    ipc = lib()
    w = small["w"]
    ctx = make_ctx(w, path="tc", max_requests=2)
    try:
        load_workload(ctx, w, chunk=300)
        code, mask = query_shares_gpu(w, small["qc"], small["qm"])
        args = ([code[j] for j in range(3)], [mask[j] for j in range(3)], w.Q, 1)
        ra = ipc.submit_queries(ctx, *args)
        rb = ipc.submit_queries(ctx, *args)
        with pytest.raises(ipc.IpcError) as e:
            ipc.submit_queries(ctx, *args)
        assert e.value.rc == ipc.IPC_EAGAIN
        ipc.ipc_release(ctx, ra)
        rc_ = ipc.submit_queries(ctx, *args)
        for rid in (rb, rc_):
            sh = np.zeros((3, w.Q), np.uint8)
            ipc.fetch_bit_shares(ctx, rid, sh, w.Q, 60000)
            assert (sh == _oracle_shares(small, rid)).all()
            ipc.ipc_release(ctx, rid)
    finally:
        ipc.ipc_destroy(ctx)


def test_admission_beyond_device_memory_is_enomem(torch, small):
    """Request slots (context) and a column pool (serving) larger than the device are refused
    with IPC_ENOMEM, without touching the resident database."""
    ipc = lib()
    w = small["w"]
    ctx = make_ctx(w, path="tc", max_queries=200000, max_requests=64)
    try:
        load_workload(ctx, w, chunk=300)
        code, mask = query_shares_gpu(w, small["qc"], small["qm"])
        with pytest.raises(ipc.IpcError) as e:
            ipc.submit_queries(ctx, [code[j] for j in range(3)], [mask[j] for j in range(3)], w.Q, 1)
        assert e.value.rc == ipc.IPC_ENOMEM
        assert ipc.ipc_db_rows(ctx) == w.s
        with pytest.raises(ipc.IpcError) as e:
            ipc.ipc_serve_start(ctx, pool_queries=10_000_000, variant=0)
        assert e.value.rc == ipc.IPC_ENOMEM
    finally:
        ipc.ipc_destroy(ctx)


def test_serving_pending_queue_full_is_eagain(torch):
    """A serving loop with one query slot and room for one waiting request: while the first
    request runs and the second waits, a third is refused with IPC_EAGAIN; the first two
    complete with the oracle's bits."""
    ipc = lib()
    w = synth.Workload("fail3", s=65536, Q=3, planted=1, seed=0xFA13)
    ctx = make_ctx(w, path="tc", max_queries=1)
    try:
        load_workload(ctx, w, chunk=32768)
        qc, qm = w.query_bits()
        code, mask = query_shares_gpu(w, qc, qm)
        hc = [code[j].cpu().numpy() for j in range(3)]
        hm = [mask[j].cpu().numpy() for j in range(3)]
        ipc.ipc_serve_start(ctx, pool_queries=1, max_pending=1, variant=0)
        sub = lambda q: ipc.ipc_serve_submit(ctx, [np.ascontiguousarray(hc[j][q:q + 1]) for j in range(3)],
                                            [np.ascontiguousarray(hm[j][q:q + 1]) for j in range(3)], 1)
        ra, rb = sub(0), sub(1)
        with pytest.raises(ipc.IpcError) as e:
            sub(2)
        assert e.value.rc == ipc.IPC_EAGAIN
        dc, dm = w.db_bits()
        match, _, _ = oracle.plain_match(oracle.iris_geom(), qc, qm, dc, dm)
        for q, rid in ((0, ra), (1, rb)):
            b = np.zeros(1, np.uint8)
            ipc.fetch_match_bits(ctx, rid, b, 1, 600000)
            assert b[0] == match[q]
        ipc.ipc_serve_stop(ctx)
    finally:
        ipc.ipc_destroy(ctx)


def test_flipped_message_bit_changes_the_result_undetected(torch):
    """Semi-honest security (Sec. 2): a bit flipped in one party's reshared dot product (an A4
    message) is not detected; the comparison and OR tree run on the tampered message exactly as
    the oracle does, and the opened result changes. One comparison matches (dot = ml = 5,000);
    flipping bit 14 of party 1's component subtracts 2^14 from the dot, so no row matches."""
    ipc = lib()
    rng = np.random.default_rng(0xF1B)
    Q, R, s = 1, 31, 1000
    N, ldz = Q * R, 1000
    ml = np.full((N, s), 5000, np.int64)
    dot = np.zeros((N, s), np.int64)
    dot[7, 321] = 5000

    def share(v):
        c0 = rng.integers(0, 65536, size=v.shape)
        c1 = rng.integers(0, 65536, size=v.shape)
        return np.stack([c0, c1, (v - c0 - c1) & 0xFFFF]).astype(np.uint16)

    zc_h, zm_h = share(dot), share(ml)
    seeds = (0x5EED0, 0x5EED1, 0x5EED2)
    cfg = oracle.mpc_cfg(seeds, req=3)
    tags = np.zeros((N, 2), np.uint32)
    tags[:, 0] = 3
    tags[:, 1] = np.arange(N)
    dtags = torch.from_numpy(tags.view(np.int32)).cuda()
    zm = torch.from_numpy(zm_h.view(np.int16)).cuda()

    def run(zc_np):
        zc = torch.from_numpy(zc_np.view(np.int16).copy()).cuda()
        roots = torch.zeros((3, N, 1), dtype=torch.int32, device="cuda")
        bits = torch.zeros((3, Q), dtype=torch.uint8, device="cuda")
        ipc.ipc_compare([zc[j] for j in range(3)], [zm[j] for j in range(3)], ldz, N, s, 0, dtags, seeds, 16384, 5,
                        roots, 1)
        ipc.ipc_or_finalize(roots, 1, 1, 5, Q, R, dtags, seeds, bits)
        torch.cuda.synchronize()
        ipc.ipc_status()
        msb = np.zeros((3, N, s), np.uint8)
        for n in range(N):
            for i in range(s):
                msb[:, n, i] = oracle.mpc_compare(cfg, zc_np[:, n, i], zm_h[:, n, i], 0, n, i)[0]
        want = oracle.or_tree(cfg, msb, 0)
        return bits.cpu().numpy()[:, 0], want

    got, want = run(zc_h)
    assert (got == want).all() and oracle.reconstruct_bits(got[:, None])[0] == 1
    tampered = zc_h.copy()
    tampered[1, 7, 321] ^= 1 << 14
    got_t, want_t = run(tampered)
    assert (got_t == want_t).all() and oracle.reconstruct_bits(got_t[:, None])[0] == 0
