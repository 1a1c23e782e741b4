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
