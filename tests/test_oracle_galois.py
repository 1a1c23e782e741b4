"""Pins of the oracle's Galois-ring Shamir dot products (Sec. 4.3.2).

GR = Z_{2^16}[X]/(X^2 - X - 1). The ring arithmetic is checked against an independent model
(multiplication by a0 + a1 X as the 2 x 2 integer matrix a0 I + a1 M, M the companion matrix of
X^2 - X - 1), the unit criterion against the residue field F_4, the Lagrange coefficients by
interpolating polynomials of degree <= 2, the sharing by reconstruction, and the dot products
and the whole protocol against the plaintext Alg. 1."""
import numpy as np
import pytest

import oracle
import synth

M = np.array([[0, 1], [1, 1]], dtype=np.int64)  # x (1, X) basis: X*1 = X, X*X = 1 + X
MOD = 1 << 16


def mat(a):
    return (int(a[0]) * np.eye(2, dtype=np.int64) + int(a[1]) * M) % MOD


def elem(A):
    return np.array([A[0, 0] % MOD, A[1, 0] % MOD], dtype=np.uint16)  # A applied to 1


def mm(*mats):
    out = np.eye(2, dtype=np.int64)
    for A in mats:
        out = (out @ A) % MOD
    return out


def test_gr_mul_is_the_matrix_ring_product():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        a, b = rng.integers(0, MOD, 2), rng.integers(0, MOD, 2)
        assert (oracle.gr_mul(a, b) == elem(mm(mat(a), mat(b)))).all()
    # X^2 = X + 1 (the defining relation) and the identity
    assert oracle.gr_mul([0, 1], [0, 1]).tolist() == [1, 1]
    assert oracle.gr_mul([1, 0], [123, 456]).tolist() == [123, 456]


def test_units_are_the_elements_nonzero_mod_2():
    # GR / 2GR = F_2[X]/(X^2 + X + 1) = F_4, so a is a unit iff (a0, a1) mod 2 != (0, 0)
    rng = np.random.default_rng(2)
    for _ in range(3000):
        a = rng.integers(0, MOD, 2)
        inv = oracle.gr_inv(a)
        unit = bool((a[0] | a[1]) & 1)
        assert (inv is not None) == unit
        if unit:
            assert (elem(mm(mat(a), mat(inv))) == [1, 0]).all()


def test_points_are_exceptional_and_lagrange_interpolates_at_zero():
    alpha = oracle.gr_points()
    lam = oracle.gr_lagrange()
    for i in range(3):
        assert (alpha[i] & 1).any()  # non-zero mod 2: a unit
        for j in range(i + 1, 3):
            assert oracle.gr_inv((alpha[j].astype(np.int64) - alpha[i]) % MOD) is not None
    # sum_p lambda_p alpha_p^k = [k == 0] for k = 0, 1, 2
    for k in range(3):
        tot = np.zeros((2, 2), np.int64)
        for p in range(3):
            tot = (tot + mm(mat(lam[p]), *([mat(alpha[p])] * k))) % MOD
        expect = np.eye(2, dtype=np.int64) if k == 0 else np.zeros((2, 2), np.int64)
        assert (tot == expect).all(), k
    # random polynomials of degree 2 over GR: interpolation gives the constant term
    rng = np.random.default_rng(3)
    for _ in range(200):
        f = [rng.integers(0, MOD, 2) for _ in range(3)]
        tot = np.zeros((2, 2), np.int64)
        for p in range(3):
            A = mat(alpha[p])
            fa = (mat(f[0]) + mm(mat(f[1]), A) + mm(mat(f[2]), A, A)) % MOD
            tot = (tot + mm(mat(lam[p]), fa)) % MOD
        assert (elem(tot) == f[0]).all()


def test_sharing_reconstructs_from_any_two_shares():
    rng = np.random.default_rng(4)
    l, n = 64, 5
    cb = rng.integers(0, 2**63, size=(n, 1), dtype=np.int64).view(np.uint64)
    mb = rng.integers(0, 2**63, size=(n, 1), dtype=np.int64).view(np.uint64)
    code, mask = oracle.encode_share_galois(cb, mb, l, 0xC11E, 0)
    alpha = oracle.gr_points()
    bits = lambda w, b: int((int(w[b >> 6]) >> (b & 63)) & 1)
    for r in range(n):
        for e in range(l // 2):
            want_c = [(bits(mb[r], 2 * e + t) - 2 * (bits(cb[r], 2 * e + t) & bits(mb[r], 2 * e + t))) % MOD
                      for t in range(2)]
            want_m = [bits(mb[r], 2 * e + t) for t in range(2)]
            for shares, want in ((code, want_c), (mask, want_m)):
                s = [shares[p, r, 2 * e:2 * e + 2] for p in range(3)]
                for j, k in ((0, 1), (0, 2), (1, 2)):
                    # degree 1: g = (alpha_k s_j - alpha_j s_k) / (alpha_k - alpha_j)
                    num = (mm(mat(alpha[k]), mat(s[j])) - mm(mat(alpha[j]), mat(s[k]))) % MOD
                    den = oracle.gr_inv((alpha[k].astype(np.int64) - alpha[j]) % MOD)
                    assert (elem(mm(num, mat(den))) == want).all()
    # one party's share alone is uniform: coefficient means near 2^15
    assert abs(code[1].astype(np.float64).mean() - 32767.5) < 2500


@pytest.mark.parametrize("seed", [5, 6])
def test_dot_components_sum_to_the_plain_dot(seed):
    rng = np.random.default_rng(seed)
    l = 256
    cb = rng.integers(0, 2**63, size=(2, l // 64), dtype=np.int64).view(np.uint64)
    mb = rng.integers(0, 2**63, size=(2, l // 64), dtype=np.int64).view(np.uint64)
    code, mask = oracle.encode_share_galois(cb, mb, l, 0xABC, 0)
    cfg = oracle.mpc_cfg(req=3)
    ml, hd = oracle.plain_pair(cb[0], mb[0], cb[1], mb[1])
    zc = oracle.mpc_dot_galois(cfg, code[:, 0], code[:, 1], 1, 2, 7, 0)
    zm = oracle.mpc_dot_galois(cfg, mask[:, 0], mask[:, 1], 1, 2, 7, 1)
    assert int(oracle.reconstruct_u16(zc)) == (ml - 2 * hd) % MOD
    assert int(oracle.reconstruct_u16(zm)) == ml


def test_galois_protocol_equals_alg1():
    w = synth.Workload("galois", s=40, Q=3, planted=2, seed=0x6A10)
    g = oracle.iris_geom()
    dc, dm = w.db_bits()
    qc, qm = w.query_bits()
    dbc, dbm = oracle.encode_share_galois(dc, dm, w.l, w.db_share_seed, 0)
    qsc, qsm = oracle.encode_share_galois(qc, qm, w.l, w.q_share_seed, 1)
    match, ml, hd = oracle.plain_match(g, qc, qm, dc, dm, distances=True)
    ref = oracle.mpc_match_galois(oracle.mpc_cfg(w.prf_seeds, req=9), g, dbc, dbm, qsc, qsm, want_z=True)
    assert (oracle.reconstruct_bits(ref["bits"]) == match).all()
    assert match.sum() == w.planted
    n = w.Q * w.R
    assert (oracle.reconstruct_u16(ref["z_mask"]) == ml.reshape(n, -1)).all()
    assert (oracle.reconstruct_u16(ref["z_code"]) == ((ml - 2 * hd).reshape(n, -1) & 0xFFFF)).all()
