"""Pins of the oracle's protocol 1 (Sec. 4, Alg. 2: shared codes, public masks): the 16-bit
MSB comparison against Alg. 1's strict rule over every boundary, its gate count and depth
(29 ANDs, 15 rounds, Sec. 4.3.1), and the whole protocol against Alg. 1."""
import numpy as np
import pytest

import oracle
import synth


def _share16(rng, v):
    a, b = rng.integers(0, 1 << 16, 2)
    return np.array([a, b, (v - a - b) & 0xFFFF], dtype=np.uint16)


def test_comparison_is_alg1_rule_on_every_boundary():
    rng = np.random.default_rng(31)
    cfg = oracle.mpc_cfg(req=2)
    cases = []
    for ml in list(range(0, 40)) + [12799, 12800] + list(rng.integers(0, 12801, 60)):
        q4 = ml // 4
        for dot in {q4 - 1, q4, q4 + 1, q4 + 2, -ml, ml, 0}:
            if -ml <= dot <= ml:
                cases.append((int(ml), int(dot)))
    for ml, dot in cases:
        msb = oracle.mpc_compare_plain(cfg, _share16(rng, dot & 0xFFFF), ml)
        assert int(oracle.reconstruct_bits(msb)) == int(4 * dot > ml), (ml, dot)


def test_gate_count_and_depth():
    st = oracle.Stats()
    oracle.mpc_compare_plain(oracle.mpc_cfg(), np.array([1, 2, 3], np.uint16), 100, stats=st)
    d = st.as_dict()
    assert d["and_msb"] == 29 and d["depth_msb"] == 15


@pytest.mark.parametrize("galois", [False, True])
def test_protocol1_equals_alg1(galois):
    w = synth.Workload("p1", s=60, Q=3, planted=2, seed=0x9A51)
    g = oracle.iris_geom()
    dc, dm = w.db_bits()
    qc, qm = w.query_bits()
    enc = oracle.encode_share_galois if galois else oracle.encode_share
    dbc, _ = enc(dc, dm, w.l, w.db_share_seed, 0)
    qsc, _ = enc(qc, qm, w.l, w.q_share_seed, 1)
    match, ml, hd = oracle.plain_match(g, qc, qm, dc, dm, distances=True)
    ref = oracle.mpc_match_plain(oracle.mpc_cfg(w.prf_seeds, req=5), g, dbc, dm, qsc, qm, galois=galois,
                                 want_z=True)
    n = w.Q * w.R
    assert (ref["ml"] == ml.reshape(n, -1)).all()
    assert (oracle.reconstruct_u16(ref["z_code"]) == ((ml - 2 * hd).reshape(n, -1) & 0xFFFF)).all()
    assert (oracle.reconstruct_bits(ref["bits"]) == match).all() and match.sum() == w.planted
