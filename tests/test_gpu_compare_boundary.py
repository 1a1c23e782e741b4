"""GPU parity of the headline comparison kernel (MPCLift: Lift, threshold, MSB, OR tree) on
the threshold boundary, against the oracle share for share.

Alg. 3 with a/b = 1/4 (Lemma 2) matches when 4 dot > ml, i.e. when v = a ml - 2^16 dot < 0.
The cells below sit on that edge: v = 0 (4 dot = ml, no match), v = -2^14 (4 dot = ml + 1,
match), v = +2^14 and the rest of the neighbourhood, ml = 0 with dot = 0, ml at the ends of
Z_2^16, and ml share triples whose integer sum carries 0, 1 or 2 times past 2^16 -- the three
cases the Lift's BitExtract of bits 17 and 16 and its BitInject must undo (Sec. 5.1, App. D).
"""
import numpy as np
import pytest

import oracle
from gpu_common import lib, tags_for, torch_mod

pytestmark = pytest.mark.gpu

SEEDS = (0x5EED0, 0x5EED1, 0x5EED2)
REQ = 11
THR_A = 16384
Q, R = 2, 31
S = 1024 + 3 * 32 + 9   # one full 1,024-row OR block and a ragged one (four words and 9 rows)
LDZ = (S + 7) // 8 * 8
M16 = 65536


def _boundary_pairs():
    """(ml, dot) on and around 4 dot = ml, for ml in 0..39, the largest code lengths and the
    ends of Z_2^16; dot is kept in int16 and |v| = 2^14 |ml - 4 dot| below 2^31 (Lemma 2)."""
    mls = list(range(40)) + [12799, 12800, 2**15 - 1, 2**15, 2**15 + 1, M16 - 4, M16 - 3, M16 - 1]
    out = []
    for ml in mls:
        f = ml // 4
        for dot in sorted({f - 1, f, f + 1, -ml, ml, 0}):
            if -2**15 <= dot < 2**15 and abs(ml - 4 * dot) < 2**17:
                out.append((ml, dot))
    return out


def _ml_triple(rng, ml, carry):
    """Three components in [0, 2^16) summing, as integers, to ml + carry * 2^16."""
    total = ml + carry * M16
    assert 0 <= total <= 3 * (M16 - 1)
    a = int(rng.integers(max(0, total - 2 * (M16 - 1)), min(M16 - 1, total) + 1))
    b = int(rng.integers(max(0, total - a - (M16 - 1)), min(M16 - 1, total - a) + 1))
    t = [a, b, total - a - b]
    rng.shuffle(t)
    return t


def _dot_triple(rng, dot):
    a, b = (int(x) for x in rng.integers(0, M16, 2))
    return [a, b, (dot - a - b) % M16]


def _workload():
    """Columns of query 0 hold every boundary pair under each Lift carry, then random ml with
    dot = floor(ml / 4) + {-1, 0, 1}; query 1 holds only cells with 4 dot <= ml (no match, v = 0
    included), so its opened OR bit must be 0."""
    rng = np.random.default_rng(0xB0DE)
    N = Q * R
    ml = np.zeros((N, S), np.int64)
    dot = np.zeros((N, S), np.int64)
    carry = np.zeros((N, S), np.int64)
    pairs = _boundary_pairs()
    crafted = [(m, d, c) for (m, d) in pairs for c in (0, 1, 2) if m + c * M16 <= 3 * (M16 - 1)]
    for q in range(Q):
        cells = crafted if q == 0 else [t for t in crafted if 4 * t[1] <= t[0]]
        cols = range(q * R, (q + 1) * R)
        flat = [(n, i) for n in cols for i in range(S)]
        order = rng.permutation(len(flat))
        for k, idx in enumerate(order):
            n, i = flat[idx]
            if k < len(cells):
                ml[n, i], dot[n, i], carry[n, i] = cells[k]
            else:
                m = int(rng.integers(0, 12801))
                d = m // 4 + (int(rng.integers(-1, 2)) if q == 0 else -int(rng.integers(0, 3)))
                ml[n, i], dot[n, i], carry[n, i] = m, d, int(rng.integers(0, 3))
    zc = np.zeros((3, N, LDZ), np.uint16)
    zm = np.zeros((3, N, LDZ), np.uint16)
    for n in range(N):
        for i in range(S):
            zc[:, n, i] = _dot_triple(rng, int(dot[n, i]))
            zm[:, n, i] = _ml_triple(rng, int(ml[n, i]), int(carry[n, i]))
    return ml, dot, carry, zc, zm


@pytest.fixture(scope="module")
def case():
    torch = torch_mod()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ml, dot, carry, zc, zm = _workload()
    cfg = oracle.mpc_cfg(SEEDS, req=REQ, thr_a=THR_A)
    N = Q * R
    msb = np.zeros((3, N, S), np.uint8)
    for n in range(N):
        q, rho = divmod(n, R)
        for i in range(S):
            msb[:, n, i] = oracle.mpc_compare(cfg, zc[:, n, i], zm[:, n, i], q, rho, i)[0]
    bits = np.stack([oracle.or_tree(cfg, msb[:, q * R:(q + 1) * R], q) for q in range(Q)], axis=1)
    return dict(ml=ml, dot=dot, carry=carry, zc=zc, zm=zm, msb=msb, bits=bits, torch=torch)


def test_boundary_cells_cover_every_lift_carry(case):
    """The crafted grid reaches v = 0, v = -2^14, ml = 0 with dot = 0, and every carry."""
    ml, dot, carry = case["ml"], case["dot"], case["carry"]
    v = ml - 4 * dot
    q0 = slice(0, R)
    assert (v[q0] == 0).any() and (v[q0] == -1).any() and (v[q0] == 1).any()
    assert ((ml[q0] == 0) & (dot[q0] == 0)).any()
    for c in (0, 1, 2):
        assert ((carry == c) & (v == 0)).any() and ((carry == c) & (v == -1)).any()
    assert (ml == M16 - 1).any() and (ml == 2**15).any()


def test_oracle_opens_alg1_rule_on_the_boundary(case):
    """Alg. 1's strict rule (hd / ml < 3/8, i.e. 4 dot > ml; ml = 0 never matches), from the
    oracle's opened MSBs, on every cell; and the OR over each query."""
    opened = case["msb"][0] ^ case["msb"][1] ^ case["msb"][2]
    assert (opened == (4 * case["dot"] > case["ml"])).all()
    assert oracle.reconstruct_bits(case["bits"]).tolist() == [1, 0]


@pytest.mark.parametrize("log2_block_words", [5, 2])
def test_mpclift_compare_matches_oracle_on_the_boundary(case, log2_block_words):
    torch = case["torch"]
    ipc = lib()
    N, p = Q * R, log2_block_words
    zc = torch.from_numpy(case["zc"].view(np.int16)).cuda()
    zm = torch.from_numpy(case["zm"].view(np.int16)).cuda()
    tags = torch.from_numpy(tags_for(REQ, Q, R).view(np.int32)).cuda()
    nb = (S + (32 << p) - 1) >> (5 + p)
    roots = torch.zeros((3, N, nb), dtype=torch.int32, device="cuda")
    msb = torch.zeros((3, N, S), dtype=torch.uint8, device="cuda")
    ipc.ipc_compare([zc[j] for j in range(3)], [zm[j] for j in range(3)], LDZ, N, S, 0, tags, SEEDS, THR_A, p, roots,
                    nb, msb, S)
    bits = torch.zeros((3, Q), dtype=torch.uint8, device="cuda")
    ipc.ipc_or_finalize(roots, nb, nb, p, Q, R, tags, SEEDS, bits)
    torch.cuda.synchronize()
    ipc.ipc_status()
    got = msb.cpu().numpy()
    bad = np.argwhere((got != case["msb"]).any(axis=0))
    assert bad.size == 0, [(int(n), int(i), int(case["ml"][n, i]), int(case["dot"][n, i]), int(case["carry"][n, i]))
                           for n, i in bad[:8]]
    assert (bits.cpu().numpy() == case["bits"]).all()


def test_noalloc_entry_matches_oracle_on_the_boundary(case):
    """The same cells through the allocation-free entry point, on a non-default stream."""
    torch = case["torch"]
    ipc = lib()
    zc = torch.from_numpy(case["zc"].view(np.int16)).cuda()
    zm = torch.from_numpy(case["zm"].view(np.int16)).cuda()
    tags = torch.from_numpy(tags_for(REQ, Q, R).view(np.int32)).cuda()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    out = torch.full((3, Q), 9, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(st):
        ipc.ipc_compare_or_noalloc([zc[j] for j in range(3)], [zm[j] for j in range(3)], LDZ, Q, R, S, tags, SEEDS,
                                   THR_A, out, stream=st)
    st.synchronize()
    ipc.ipc_status()
    assert (out.cpu().numpy() == case["bits"]).all()
