"""Pins of the oracle's lifting variants (Sec. 5.1, Sec. 6.2 Table 2): ConstLift (ml computed
over Z_2^32, dot over Z_2^16 lifted for free) and NoLift (both over Z_2^32).

Pinned by what the mathematics fixes: the Z_2^32 encoding reconstructs the T/U/F table and
agrees with the 16-bit one modulo 2^16; the Z_2^32 dot reconstructs the plaintext dot and,
on encoded iris codes, Alg. 1's distances; the lift-free comparison is the Alg. 3 rule on
every reachable ml with dots on each side of the threshold, for b = 2^16 and for another
16-bit b; the comparison uses Table 2's 61 ANDs and no Lift; whole matches equal Alg. 1.
"""
import numpy as np
import pytest

import oracle
import synth

L = 12800


def _split32(rng, v):
    a, b = (int(t) for t in rng.integers(0, 1 << 32, 2, dtype=np.uint64))
    return [a, b, (v - a - b) & 0xFFFFFFFF]


def _split16(rng, v):
    a, b = (int(t) for t in rng.integers(0, 1 << 16, 2))
    return [a, b, (v - a - b) & 0xFFFF]


def _rec32(sh):
    return (np.asarray(sh).astype(np.uint64).sum(axis=0) & 0xFFFFFFFF).astype(np.uint32)


def test_encode_share32_reconstructs_the_encoding():
    rng = np.random.default_rng(40)
    n, l = 5, 256
    cb = rng.integers(0, 2**63, (n, l // 64), dtype=np.uint64)
    mb = rng.integers(0, 2**63, (n, l // 64), dtype=np.uint64)
    code, mask = oracle.encode_share32(cb, mb, l, 0xC11E, 0)
    bits = lambda w: np.unpackbits(w.view(np.uint8), axis=1, bitorder="little")[:, :l].astype(np.int64)
    c, m = bits(cb), bits(mb)
    # masked bit: T (c=1, m=1) -> -1, U (m=0) -> 0, F (c=0, m=1) -> +1, read in Z_2^32
    expect = (m - 2 * (c & m)) & 0xFFFFFFFF
    assert (_rec32(code).astype(np.int64) == expect).all()
    assert (_rec32(mask).astype(np.int64) == m).all()
    assert set(np.unique(expect).tolist()) <= {0, 1, 0xFFFFFFFF}
    # modulo 2^16 it is the 16-bit encoding's secret
    c16, m16 = oracle.encode_share(cb, mb, l, 0xC11E, 0)
    assert (_rec32(code) & 0xFFFF == oracle.reconstruct_u16(c16)).all()
    assert (_rec32(mask) & 0xFFFF == oracle.reconstruct_u16(m16)).all()
    # the random components use the full 32 bits (top bit about half the time)
    top = (code[0] >> 31).mean()
    assert 0.4 < top < 0.6 and (code[1] >> 16).max() > 0


def test_dot32_reconstructs_plaintext_dot_and_zero_shares_cancel():
    rng = np.random.default_rng(41)
    l = 512
    for trial in range(20):
        x = rng.integers(-(2**31), 2**31, l, dtype=np.int64)
        y = rng.integers(-(2**31), 2**31, l, dtype=np.int64)
        xs = np.stack(_split_vec(rng, x))
        ys = np.stack(_split_vec(rng, y))
        want = int(np.sum((x.astype(object) * y.astype(object)))) & 0xFFFFFFFF
        z1 = oracle.mpc_dot32(oracle.mpc_cfg(req=1), xs, ys, 0, trial, 3, 0)
        z2 = oracle.mpc_dot32(oracle.mpc_cfg(req=2), xs, ys, 0, trial, 3, 0)
        assert int(_rec32(z1)) == want == int(_rec32(z2))
        assert (z1 != z2).any()   # re-randomised differently, same secret


def _split_vec(rng, v):
    a = rng.integers(0, 2**32, v.shape, dtype=np.uint64)
    b = rng.integers(0, 2**32, v.shape, dtype=np.uint64)
    c = (v.astype(np.uint64) - a - b) & np.uint64(0xFFFFFFFF)
    return [a.astype(np.uint32), b.astype(np.uint32), c.astype(np.uint32)]


def test_dot32_on_encoded_irises_gives_alg1_distances():
    w = synth.Workload("d32", s=6, Q=1, planted=1, seed=0x3232)
    g = oracle.iris_geom()
    dc, dm = w.db_bits()
    qc, qm = w.query_bits()
    _, ml, hd = oracle.plain_match(g, qc, qm, dc, dm, distances=True)
    xc, xm = oracle.encode_share32(dc, dm, w.l, 1, 0)
    yc, ym = oracle.encode_share32(qc, qm, w.l, 2, 1)
    cfg = oracle.mpc_cfg(req=9)
    for rho in (0, 15, 30):
        shift = g.rot_lo + rho
        ryc = np.stack([_rot32(g, yc[j, 0], shift) for j in range(3)])
        rym = np.stack([_rot32(g, ym[j, 0], shift) for j in range(3)])
        for i in range(w.s):
            dot = int(_rec32(oracle.mpc_dot32(cfg, xc[:, i], ryc, 0, rho, i, 0)))
            mll = int(_rec32(oracle.mpc_dot32(cfg, xm[:, i], rym, 0, rho, i, 1)))
            assert mll == ml[0, rho, i]
            assert dot == (int(ml[0, rho, i]) - 2 * int(hd[0, rho, i])) & 0xFFFFFFFF


def _rot32(g, v, shift):
    # rotation of a u32 vector through two u16 halves (the 16-bit rotation is pinned elsewhere)
    lo = oracle.rotate_u16(g, (v & 0xFFFF).astype(np.uint16), shift).astype(np.uint32)
    hi = oracle.rotate_u16(g, (v >> 16).astype(np.uint16), shift).astype(np.uint32)
    return lo | (hi << 16)


def _cases(rng, n):
    out = []
    for ml in list(range(0, 64)) + [L - 1, L] + [int(t) for t in rng.integers(0, L + 1, n)]:
        q4 = ml // 4
        for dot in {q4 - 1, q4, q4 + 1, -ml, ml, 0, int(rng.integers(-ml, ml + 1))}:
            if -ml <= dot <= ml:
                out.append((ml, dot))
    return out


@pytest.mark.parametrize("mode", [oracle.LIFT_CONST, oracle.LIFT_NONE])
def test_liftfree_compare_is_alg3_rule(mode):
    rng = np.random.default_rng(42)
    cfg = oracle.mpc_cfg((5, 6, 7), req=4)
    st = oracle.Stats()
    for k, (ml, dot) in enumerate(_cases(rng, 300)):
        m = _split32(rng, ml)
        d = _split16(rng, dot & 0xFFFF) if mode == oracle.LIFT_CONST else _split32(rng, dot & 0xFFFFFFFF)
        msb, v = oracle.mpc_compare_liftfree(cfg, mode, d, m, 0, 1, 2, k, stats=st)
        assert int(_rec32(v)) == (16384 * ml - 65536 * dot) & 0xFFFFFFFF
        assert int(oracle.reconstruct_bits(msb)) == int(65536 * dot > 16384 * ml), (ml, dot)
    assert st.and_msb == 61 and st.depth_msb == 31 and st.and_lift == 0
    assert st.replication_errors == 0


def test_nolift_with_another_16bit_b():
    # NoLift needs no ConstLift, so b need not be a power of two: a / b = 10000 / 40000 = 1/4
    rng = np.random.default_rng(43)
    cfg = oracle.mpc_cfg((8, 9, 10), req=5, thr_a=10000)
    for k, (ml, dot) in enumerate(_cases(rng, 200)):
        msb, v = oracle.mpc_compare_liftfree(cfg, oracle.LIFT_NONE, _split32(rng, dot & 0xFFFFFFFF),
                                             _split32(rng, ml), 40000, 0, 0, k)
        assert int(_rec32(v)) == (10000 * ml - 40000 * dot) & 0xFFFFFFFF
        assert int(oracle.reconstruct_bits(msb)) == int(40000 * dot > 10000 * ml), (ml, dot)


@pytest.mark.parametrize("mode", [oracle.LIFT_CONST, oracle.LIFT_NONE])
def test_match_lift_equals_alg1(mode):
    w = synth.Workload("lift", s=40, Q=3, planted=2, seed=0x11F7)
    g = oracle.iris_geom()
    dc, dm = w.db_bits()
    qc, qm = w.query_bits()
    match, ml, hd = oracle.plain_match(g, qc, qm, dc, dm, distances=True)
    c32, m32 = oracle.encode_share32(dc, dm, w.l, w.db_share_seed, 0)
    qc32, qm32 = oracle.encode_share32(qc, qm, w.l, w.q_share_seed, 1)
    if mode == oracle.LIFT_CONST:
        dbc, _ = oracle.encode_share(dc, dm, w.l, w.db_share_seed, 0)
        qsc, _ = oracle.encode_share(qc, qm, w.l, w.q_share_seed, 1)
    else:
        dbc, qsc = c32, qc32
    ref = oracle.mpc_match_lift(oracle.mpc_cfg(w.prf_seeds, req=3), g, mode, dbc, m32, qsc, qm32, want_z=True)
    n = w.Q * w.R
    assert (_rec32(ref["z_mask"]) == ml.reshape(n, -1)).all()
    dot = (ml - 2 * hd).reshape(n, -1)
    if mode == oracle.LIFT_CONST:
        assert (oracle.reconstruct_u16(ref["z_code"]) == (dot & 0xFFFF)).all()
    else:
        assert (_rec32(ref["z_code"]).astype(np.int64) == (dot.astype(np.int64) & 0xFFFFFFFF)).all()
    assert (oracle.reconstruct_bits(ref["bits"]) == match).all() and match.sum() == w.planted
    assert ref["stats"]["and_msb"] == 61 and ref["stats"]["and_lift"] == 0
