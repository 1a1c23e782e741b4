"""Pins of the CPU oracle against what the paper and mathematics fix (no GPU).

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms (App. B, App. C, Lemma 2), textbook or
library routines, brute force, invariants, or counts printed in the paper.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.spatial.distance as ssd

import oracle
import synth
from conftest import read_golden

L = 12800


def _bits(rng, n, l, p=0.5):
    return rng.random((n, l)) < p


# ---------------------------------------------------------------- PRF ----------

def test_philox_known_answers():
    rows = read_golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox(v[0:2], v[2:6])
        assert [int(x) for x in out] == v[6:10]


# ---------------------------------------------------- encoding and sharing -------

def test_masked_bit_encoding_table():
    # Sec. 4.1.1: (T, U, F) = (-1, 0, 1); T = code and mask set, F = mask set code clear, U = mask clear.
    code = np.array([[0, 1, 0, 1] * 16], dtype=bool)
    mask = np.array([[0, 0, 1, 1] * 16], dtype=bool)
    cs, ms = oracle.encode_share(synth.pack_bits(code), synth.pack_bits(mask), 64, 7, 0)
    val = oracle.reconstruct_u16(cs)[0].astype(np.int32)
    val = np.where(val >= 32768, val - 65536, val)
    assert list(val[:4]) == [0, 0, 1, -1]
    assert list(oracle.reconstruct_u16(ms)[0][:4]) == [0, 0, 1, 1]


def test_sharing_reconstructs_and_looks_uniform():
    rng = np.random.default_rng(1)
    c, m = _bits(rng, 8, 256), _bits(rng, 8, 256, 0.9)
    cs, ms = oracle.encode_share(synth.pack_bits(c), synth.pack_bits(m), 256, 99, 1, idx0=5)
    enc = (m.astype(np.int64) - 2 * (c & m)) & 0xFFFF
    assert (oracle.reconstruct_u16(cs) == enc).all()
    assert (oracle.reconstruct_u16(ms) == m).all()
    # each single component is uniform over Z_2^16 (mean 32767.5, sd 18918/sqrt(n))
    for comp in (cs[0], cs[1], cs[2], ms[0]):
        assert abs(comp.mean() - 32767.5) < 6 * 18918 / np.sqrt(comp.size)
    # different client seeds give different shares of the same secret
    cs2, _ = oracle.encode_share(synth.pack_bits(c), synth.pack_bits(m), 256, 100, 1, idx0=5)
    assert (cs2[0] != cs[0]).mean() > 0.99
    assert (oracle.reconstruct_u16(cs2) == enc).all()


# -------------------------------------------------------------- rotation --------

def test_rotation_hand_example_and_group_laws():
    g = oracle.Geom(1, 4, 2, 0, 1)
    v = np.arange(8, dtype=np.uint16)          # columns (0,1) (2,3) (4,5) (6,7)
    assert list(oracle.rotate_u16(g, v, 1)) == [6, 7, 0, 1, 2, 3, 4, 5]
    gi = oracle.iris_geom()
    x = np.random.default_rng(2).integers(0, 65536, L).astype(np.uint16)
    assert (oracle.rotate_u16(gi, x, 0) == x).all()
    assert (oracle.rotate_u16(gi, x, 200) == x).all()
    a = oracle.rotate_u16(gi, oracle.rotate_u16(gi, x, 7), -3)
    assert (a == oracle.rotate_u16(gi, x, 4)).all()
    assert np.sort(oracle.rotate_u16(gi, x, -15)).tolist() == np.sort(x).tolist()


def test_rotation_bits_matches_u16():
    gi = oracle.iris_geom()
    b = _bits(np.random.default_rng(3), 1, L)
    for sh in (-15, -1, 1, 15):
        rb = synth.unpack_bits(oracle.rotate_bits(gi, synth.pack_bits(b), sh), L)[0]
        ru = oracle.rotate_u16(gi, b[0].astype(np.uint16), sh).astype(bool)
        assert (rb == ru).all()


# ------------------------------------------------------------ Alg. 1 ------------

def test_alg1_unmasked_is_scipy_hamming():
    rng = np.random.default_rng(4)
    c, C = _bits(rng, 1, L)[0], _bits(rng, 1, L)[0]
    ones = np.ones(L, bool)
    ml, hd = oracle.plain_pair(*(synth.pack_bits(v[None])[0] for v in (c, ones, C, ones)))
    assert ml == L
    assert hd == round(ssd.hamming(c, C) * L)


def test_alg1_masked_identity_app_b():
    # App. B: <c', C'> = ml - 2 hd with c' = m - 2(c & m); computed here by a plain dot of the
    # {-1,0,1} encodings, a different route from Alg. 1's popcounts.
    rng = np.random.default_rng(5)
    for _ in range(20):
        c, C = _bits(rng, 1, L)[0], _bits(rng, 1, L)[0]
        m, M = _bits(rng, 1, L, 0.9)[0], _bits(rng, 1, L, 0.9)[0]
        ml, hd = oracle.plain_pair(*(synth.pack_bits(v[None])[0] for v in (c, m, C, M)))
        ce = m.astype(np.int64) - 2 * (c & m)
        Ce = M.astype(np.int64) - 2 * (C & M)
        assert int(ce @ Ce) == ml - 2 * hd
        assert int(m.astype(np.int64) @ M) == ml


def test_alg1_special_cases():
    rng = np.random.default_rng(6)
    c, m = _bits(rng, 1, L)[0], _bits(rng, 1, L, 0.9)[0]
    p = lambda *v: synth.pack_bits(np.array(v))
    ml, hd = oracle.plain_pair(*(p(v)[0] for v in (c, m, c, m)))
    assert hd == 0 and ml == m.sum()
    ml, hd = oracle.plain_pair(*(p(v)[0] for v in (c, m, ~c, m)))
    assert hd == ml == m.sum()
    z = np.zeros(L, bool)
    ml, hd = oracle.plain_pair(*(p(v)[0] for v in (c, z, c, m)))
    assert ml == 0 and hd == 0


def _pair_with(ml, hd, l=64):
    m = np.zeros(l, bool)
    m[:ml] = True
    c = np.zeros(l, bool)
    C = np.zeros(l, bool)
    C[:hd] = True
    return c, m, C, m


@pytest.mark.parametrize("ml,hd,expect", [(8, 3, 0), (8, 2, 1), (0, 0, 0), (16, 6, 0), (16, 5, 1),
                                          (40, 15, 0), (40, 14, 1), (1, 0, 1), (1, 1, 0)])
def test_match_rule_boundaries(ml, hd, expect):
    # Alg. 1 compares hd/ml < 3/8 strictly; 3*ml = 8*hd is the boundary (no match); ml = 0 never matches.
    g = oracle.Geom(1, 16, 4, 0, 1)
    c, m, C, M = _pair_with(ml, hd)
    pk = lambda v: synth.pack_bits(v[None])
    for rule in (0, 1):
        match, mlo, hdo = oracle.plain_match(g, pk(c), pk(m), pk(C), pk(M), rule=rule, distances=True)
        assert (mlo[0, 0, 0], hdo[0, 0, 0]) == (ml, hd)
        assert match[0] == expect


def test_lemma2_msb_equals_comparison_exhaustive():
    # Lemma 2 with t = 2^32, b = 2^16, a = 16384, l = 12800: MSB(a*ml - b*dot mod 2^32) = [b*dot > a*ml]
    # for every reachable (ml, dot): 0 <= ml <= l, |dot| <= ml, dot = ml (mod 2).
    a, b = 16384, 65536
    assert b * L < 2**32 // 4 and b * L < 2**32 - 2**31
    for ml in range(0, L + 1, 7):
        dot = np.arange(-ml, ml + 1, 2, dtype=np.int64)
        v = (a * ml - b * dot) & 0xFFFFFFFF
        assert ((v >> 31) == (b * dot > a * ml)).all()


def test_alg1_ratio_equals_alg3_integer_rule_exhaustive():
    # hd/ml < 3/8 (exact rational, Alg. 1) <=> 2^16 (ml - 2 hd) > 16384 ml (Alg. 3, a/b = 1 - 2*3/8).
    assert Fraction(16384, 65536) == 1 - 2 * Fraction(3, 8)
    for ml in range(0, L + 1, 11):
        hd = np.arange(0, ml + 1, dtype=np.int64)
        r0 = (8 * hd < 3 * ml) & (ml > 0)
        r1 = 65536 * (ml - 2 * hd) > 16384 * ml
        assert (r0 == r1).all()


def test_random_pairs_never_match_planted_do():
    w = synth.Workload("t", s=64, Q=4, rot_lo=-15, R=31, planted=2, seed=11)
    g = oracle.iris_geom()
    dc, dm = w.db_bits()
    qc, qm = w.query_bits()
    match, ml, hd = oracle.plain_match(g, qc, qm, dc, dm, distances=True)
    frac = hd / np.maximum(ml, 1)
    planted = set(w.planted_set().tolist())
    for q in range(4):
        if q in planted:
            p = w.plant(q)
            rho = -p["u"] - g.rot_lo
            i = p["src"]
            assert abs(frac[q, rho, i] - 0.10) < 0.02   # 10% of the code bits flipped
            assert match[q] == 1
        else:
            assert match[q] == 0
            assert abs(frac[q].mean() - 0.5) < 0.01


# ------------------------------------------------------ MPC simulation ----------

def _rand_shares(rng, shape):
    return rng.integers(0, 65536, (3,) + shape).astype(np.uint16)


def test_mpc_dot_reconstructs_plain_dot():
    rng = np.random.default_rng(7)
    cfg = oracle.mpc_cfg((1, 2, 3), req=9)
    for vec in (0, 1):
        x, y = _rand_shares(rng, (L,)), _rand_shares(rng, (L,))
        z = oracle.mpc_dot(cfg, x, y, q=3, rho=4, i=77, vec=vec)
        xs = x.astype(np.int64).sum(0) & 0xFFFF
        ys = y.astype(np.int64).sum(0) & 0xFFFF
        assert int(z.astype(np.int64).sum()) & 0xFFFF == int(xs @ ys) & 0xFFFF


def _za(seed, req, q, rho, i, vec):
    w = oracle.philox([seed & 0xFFFFFFFF, seed >> 32], [i >> 3, (q << 5) | rho, req, (2 << 24) | vec])
    return (int(w[(i >> 1) & 3]) >> (16 * (i & 1))) & 0xFFFF


def test_mpc_dot_components_follow_aby3_rewritten_form():
    # App. C, second form: z_i = (x_i + x_{i-1})(y_i + y_{i-1}) - x_{i-1} y_{i-1} + r_i, r_i = F_i - F_{i-1}.
    rng = np.random.default_rng(8)
    seeds = (0x1111, 0x2222222222, 0x3)
    cfg = oracle.mpc_cfg(seeds, req=5)
    x, y = _rand_shares(rng, (L,)).astype(np.int64), _rand_shares(rng, (L,)).astype(np.int64)
    z = oracle.mpc_dot(cfg, x.astype(np.uint16), y.astype(np.uint16), q=1, rho=30, i=13, vec=1)
    for i in range(3):
        im = (i + 2) % 3
        r = _za(seeds[i], 5, 1, 30, 13, 1) - _za(seeds[im], 5, 1, 30, 13, 1)
        zi = int((x[i] + x[im]) @ (y[i] + y[im]) - x[im] @ y[im]) + r
        assert int(z[i]) == zi & 0xFFFF


def test_zero_shares_change_components_not_sum():
    rng = np.random.default_rng(9)
    x, y = _rand_shares(rng, (256,)), _rand_shares(rng, (256,))
    za = oracle.mpc_dot(oracle.mpc_cfg((1, 2, 3)), x, y, 0, 0, 0, 0)
    zb = oracle.mpc_dot(oracle.mpc_cfg((4, 5, 6)), x, y, 0, 0, 0, 0)
    assert (za != zb).any()
    assert int(za.astype(np.int64).sum()) & 0xFFFF == int(zb.astype(np.int64).sum()) & 0xFFFF


EDGE32 = [0, 1, 2**31 - 1, 2**31, 2**32 - 1, 2**30, 3 * 2**30, 0x7FFF0000, 0x80000001]


def _split(rng, v):
    x0, x1 = (int(t) for t in rng.integers(0, 2**32, 2, dtype=np.uint64))
    return [x0, x1, (v - x0 - x1) & 0xFFFFFFFF]


def test_bit_extract_msb_edges_and_random():
    rng = np.random.default_rng(10)
    cfg = oracle.mpc_cfg((7, 8, 9))
    vals = EDGE32 + [int(v) for v in rng.integers(0, 2**32, 3000, dtype=np.uint64)]
    for k, v in enumerate(vals):
        x = _split(rng, v)
        top, below = oracle.bit_extract(cfg, x, 31, i=k)
        assert oracle.reconstruct_bits(top) == (v >> 31) & 1
        assert oracle.reconstruct_bits(below) == (v >> 30) & 1


def test_bit_extract_million_random_and_every_16bit_value():
    """MSB and the bit below it of a million random 32-bit sharings (App. D), and of every 16-bit
    value under four random share triples each (Sec. 4.3.1)."""
    rng = np.random.default_rng(15)
    cfg = oracle.mpc_cfg((7, 8, 9))
    n = 1_000_000
    v = rng.integers(0, 2**32, n, dtype=np.uint64)
    a = rng.integers(0, 2**32, (n, 2), dtype=np.uint64)
    x = np.stack([a[:, 0], a[:, 1], (v - a[:, 0] - a[:, 1]) & 0xFFFFFFFF], axis=1).astype(np.uint32)
    top, below = oracle.bit_extract_batch(cfg, x, 31, oracle.MSB_GATE0)
    assert (oracle.reconstruct_bits(top.T) == (v >> 31)).all()
    assert (oracle.reconstruct_bits(below.T) == ((v >> 30) & 1)).all()
    v16 = np.tile(np.arange(1 << 16, dtype=np.uint64), 4)
    a16 = rng.integers(0, 1 << 16, (v16.size, 2), dtype=np.uint64)
    x16 = np.stack([a16[:, 0], a16[:, 1], (v16 - a16[:, 0] - a16[:, 1]) & 0xFFFF], axis=1).astype(np.uint32)
    top16, below16 = oracle.bit_extract_batch(cfg, x16, 15)
    assert (oracle.reconstruct_bits(top16.T) == (v16 >> 15)).all()
    assert (oracle.reconstruct_bits(below16.T) == ((v16 >> 14) & 1)).all()


def test_bit_extract_counts_match_paper(golden):
    counts = {r[0]: r[1] for r in golden("paper_counts.txt")}
    cfg = oracle.mpc_cfg()
    for k in (16, 32):
        st = oracle.Stats()
        oracle.bit_extract(cfg, [5, 6, 7], k - 1, stats=st)
        assert st.and_gates == 2 * k - 3
        assert st.bits_sent[0] == st.bits_sent[1] == st.bits_sent[2] == 2 * k - 3
    st16 = oracle.Stats()
    top, _ = oracle.bit_extract(cfg, [1, 2, 3], 15, stats=st16)
    assert st16.and_gates == int(counts["msb16_and_gates"])
    assert int(counts["msb32_and_gates"]) == 61 and int(counts["msb32_rounds"]) == 31
    # Table 2: per-party communication of the 16-bit (plain mask) and 32-bit (ConstLift/NoLift) MSBs
    n = int(counts["table2_comparisons"])
    assert round(29 * n / 8 / 1000) in (int(counts["table2_plain_mask_kB"]), int(counts["table2_plain_mask_kB"]) + 1)
    assert round(61 * n / 8 / 1000) in (int(counts["table2_constlift_kB"]) - 1, int(counts["table2_constlift_kB"]))


def test_bit_extract_16bit_matches_reference_adder():
    # 16-bit sharing (Sec. 4.3.1): MSB of x0+x1+x2 mod 2^16 for every residue class of a sample.
    rng = np.random.default_rng(11)
    cfg = oracle.mpc_cfg((3, 1, 4))
    for v in list(range(0, 65536, 251)) + [32767, 32768, 65535]:
        x = [int(t) for t in rng.integers(0, 2**16, 2)]
        x.append((v - x[0] - x[1]) & 0xFFFF)
        top, _ = oracle.bit_extract(cfg, x, 15, i=v)
        assert oracle.reconstruct_bits(top) == (v >> 15) & 1


def test_lift_exhaustive_over_ml():
    # Sec. 5.1 / App. D Lift: for every ml in [0, l] and random Z_2^16 share triples the lifted
    # Z_2^32 sharing reconstructs to ml itself (carries 0, 1 and 2 all occur).
    rng = np.random.default_rng(12)
    cfg = oracle.mpc_cfg((11, 12, 13), req=2)
    st = oracle.Stats()
    carries = set()
    for ml in range(0, L + 1):
        x0, x1 = (int(t) for t in rng.integers(0, 65536, 2))
        comps = [x0, x1, (ml - x0 - x1) & 0xFFFF]
        carries.add(sum(comps) >> 16)
        _, mll, _ = oracle.mpc_compare(cfg, [0, 0, 0], comps, 0, 0, ml, stats=st)
        assert int(mll.astype(np.uint64).sum()) & 0xFFFFFFFF == ml
    assert carries == {0, 1, 2}
    assert st.replication_errors == 0
    assert st.and_lift == 33 and st.depth_lift == 17 + 2
    assert st.and_msb == 61 and st.depth_msb == 31


def test_compare_matches_rule_on_reachable_values():
    rng = np.random.default_rng(13)
    cfg = oracle.mpc_cfg((21, 22, 23), req=3)
    for k in range(4000):
        ml = int(rng.integers(0, L + 1))
        dot = int(rng.integers(-ml, ml + 1))
        if (dot - ml) % 2:
            dot += 1 if dot < ml else -1
        if k < 12:   # boundary 4*dot = ml and its neighbours
            ml = 4 * (k + 1) * 8
            dot = ml // 4 + (k % 3) - 1
        d = [int(t) for t in rng.integers(0, 65536, 2)]
        d.append((dot - d[0] - d[1]) & 0xFFFF)
        m = [int(t) for t in rng.integers(0, 65536, 2)]
        m.append((ml - m[0] - m[1]) & 0xFFFF)
        msb, _, v = oracle.mpc_compare(cfg, d, m, 1, 2, k)
        vv = int(v.astype(np.uint64).sum()) & 0xFFFFFFFF
        assert vv == (16384 * ml - 65536 * dot) & 0xFFFFFFFF
        assert oracle.reconstruct_bits(msb) == int(65536 * dot > 16384 * ml)


def test_or_tree_bruteforce_and_counts():
    rng = np.random.default_rng(14)
    cfg = oracle.mpc_cfg((31, 32, 33), req=4)
    for R, s in ((1, 1), (1, 32), (3, 33), (2, 70), (5, 100)):
        G = (s + 31) // 32
        for trial in range(6):
            plain = np.zeros((R, s), np.uint8)
            if trial == 1:
                plain[rng.integers(R), rng.integers(s)] = 1
            elif trial >= 2:
                plain = (rng.random((R, s)) < 0.02 * trial).astype(np.uint8)
            a, b = rng.integers(0, 2, (2, R, s)).astype(np.uint8)
            sh = np.stack([a, b, plain ^ a ^ b])
            st = oracle.Stats()
            bit = oracle.or_tree(cfg, sh, q=trial, stats=st)
            assert oracle.reconstruct_bits(bit) == int(plain.any())
            assert st.and_gates == R * G * 32 - 1
            assert st.replication_errors == 0


@pytest.mark.parametrize("R,s", [(2, 40), (3, 70), (5, 129)])
def test_or_tree_every_single_position(R, s):
    # odd widths in both tree stages (3 rotations, 3 or 5 row words) move a word up unpaired
    cfg = oracle.mpc_cfg((1, 1, 2))
    for r in range(R):
        for i in range(s):
            plain = np.zeros((R, s), np.uint8)
            plain[r, i] = 1
            bit = oracle.or_tree(cfg, np.stack([plain, plain, plain]), q=i)
            assert oracle.reconstruct_bits(bit) == 1


def test_mpc_match_small_geometry_end_to_end():
    g = oracle.Geom(2, 8, 4, -1, 3)
    w = synth.Workload("t", s=70, Q=4, rot_lo=-1, R=3, planted=2, rows=2, cols=8, cell=4, flip=0.1, seed=5)
    dc, dm = w.db_bits()
    qc, qm = w.query_bits()
    match, ml, hd = oracle.plain_match(g, qc, qm, dc, dm, rule=1, distances=True)
    dbc, dbm = oracle.encode_share(dc, dm, w.l, w.db_share_seed, 0)
    qsc, qsm = oracle.encode_share(qc, qm, w.l, w.q_share_seed, 1)
    r = oracle.mpc_match(oracle.mpc_cfg(w.prf_seeds), g, dbc, dbm, qsc, qsm, want_z=True, want_msb=True)
    n = w.Q * w.R
    assert (oracle.reconstruct_u16(r["z_code"]) == ((ml - 2 * hd).reshape(n, w.s) & 0xFFFF)).all()
    assert (oracle.reconstruct_u16(r["z_mask"]) == ml.reshape(n, w.s)).all()
    rule = (65536 * (ml - 2 * hd).astype(np.int64) > 16384 * ml.astype(np.int64)).reshape(n, w.s)
    assert (oracle.reconstruct_bits(r["msb"]) == rule).all()
    assert (oracle.reconstruct_bits(r["bits"]) == match).all()
    assert r["stats"]["replication_errors"] == 0
    assert r["stats"]["depth_total"] == 1 + 19 + 31


def test_mpc_match_full_geometry_planted():
    w = synth.Workload("t", s=5, Q=2, planted=1, seed=21)
    g = oracle.iris_geom()
    qc, qm = w.query_bits()
    dc, dm = w.db_bits()
    match, _, _ = oracle.plain_match(g, qc, qm, dc, dm)
    dbc, dbm = oracle.encode_share(dc, dm, w.l, w.db_share_seed, 0)
    qsc, qsm = oracle.encode_share(qc, qm, w.l, w.q_share_seed, 1)
    r = oracle.mpc_match(oracle.mpc_cfg(w.prf_seeds), g, dbc, dbm, qsc, qsm)
    bits = oracle.reconstruct_bits(r["bits"])
    assert (bits == match).all()
    assert sorted(np.nonzero(bits)[0].tolist()) == w.planted_set().tolist()
