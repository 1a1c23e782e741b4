"""Pins of the oracle's both-eyes / inner-batch matching (Sec. 5.4): the OR combination by its
truth table, and the inner-batch match against the plaintext Alg. 1 over earlier persons."""
import itertools

import numpy as np
import pytest

import oracle

L = 12800


def test_or_combine_truth_table():
    rng = np.random.default_rng(11)
    combos = list(itertools.product([0, 1], repeat=4))
    P = len(combos)
    plain = np.array(combos, dtype=np.uint8).T  # [4][P]
    bits4 = np.zeros((4, 3, P), np.uint8)
    for k in range(4):
        r0 = rng.integers(0, 2, P, dtype=np.uint8)
        r1 = rng.integers(0, 2, P, dtype=np.uint8)
        bits4[k] = np.stack([r0, r1, plain[k] ^ r0 ^ r1])
    out = oracle.or_combine(oracle.mpc_cfg(req=4), bits4)
    assert (oracle.reconstruct_bits(out) == plain.max(axis=0)).all()


def _batch(rng, P, dup_of):
    """Random codes; person i copies person dup_of[i] with 10% of its code bits flipped."""
    nw = L // 64
    c = rng.integers(0, 2**63, size=(P, nw), dtype=np.int64).view(np.uint64).copy()
    m = np.full((P, nw), np.uint64(0xFFFFFFFFFFFFFFFF))
    for i, j in dup_of.items():
        flip = rng.choice(L, L // 10, replace=False)
        x = c[j].copy()
        for b in flip:
            x[b // 64] ^= np.uint64(1) << np.uint64(b % 64)
        c[i] = x
    return c, m


@pytest.mark.parametrize("galois", [False, True])
def test_inner_batch_flags_later_duplicates_only(galois):
    rng = np.random.default_rng(12)
    P = 5
    c, m = _batch(rng, P, {3: 1, 4: 3})  # 3 duplicates 1, 4 duplicates 3 (and so 1)
    g = oracle.Geom(16, 200, 4, -2, 5)
    enc = oracle.encode_share_galois if galois else oracle.encode_share
    qc, qm = enc(c, m, L, 0xBA7C, 1)
    bits = oracle.mpc_match_batch(oracle.mpc_cfg(req=21), g, qc, qm, galois=galois)
    # plaintext: person q is flagged iff some rotation matches some person p' < q (Alg. 1)
    expect = np.zeros(P, np.uint8)
    for q in range(1, P):
        match, _, _ = oracle.plain_match(g, c[q:q + 1], m[q:q + 1], c[:q], m[:q])
        expect[q] = match[0]
    assert expect.tolist() == [0, 0, 0, 1, 1]
    assert (oracle.reconstruct_bits(bits) == expect).all()
