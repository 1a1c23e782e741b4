"""The allocation-free comparison entry point gives the same bit shares as the regular one.

ipc_compare_or_noalloc exists for callers that may not allocate device memory while running
(a host framework that owns the memory pool, a service that reserves everything at start-up);
it keeps its block-root scratch in a fixed array inside the library. This file is collected
last so that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEEDS = (0x51EED0, 0x51EED1, 0x51EED2)
THR_A = 16384


def _shares(rng, values, ldz):
    """Three uniformly random additive components over Z_2^16 of `values` [N][rows], padded to ldz."""
    n, rows = values.shape
    c = np.zeros((3, n, ldz), np.uint16)
    c[0, :, :rows] = rng.integers(0, 65536, (n, rows))
    c[1, :, :rows] = rng.integers(0, 65536, (n, rows))
    c[2, :, :rows] = (values.astype(np.int64) - c[0, :, :rows] - c[1, :, :rows]) & 0xFFFF
    return c


def test_noalloc_matches_caller_allocated_path_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_04463_gb300 as ipc
    rng = np.random.default_rng(2024)
    Q, R, rows = 3, 31, 5000            # five 1024-row blocks, the last one ragged
    ldz = 5008
    N = Q * R
    ml = np.full((N, rows), 10000, np.int64)
    dot = np.full((N, rows), 2000, np.int64)          # 4 * 2000 < 10000: no match
    dot[0 * R + 7, 4321] = 3000                        # 4 * 3000 > 10000: query 0 matches
    dot[2 * R + 30, 17] = 3000                         # query 2 matches
    zc = torch.from_numpy(_shares(rng, dot & 0xFFFF, ldz).view(np.int16)).cuda()
    zm = torch.from_numpy(_shares(rng, ml, ldz).view(np.int16)).cuda()
    tags = np.zeros((N, 2), np.uint32)
    for q in range(Q):
        for rho in range(R):
            tags[q * R + rho] = (9, (q << 5) | rho)
    tags = torch.from_numpy(tags.view(np.int32)).cuda()
    zcs, zms = [zc[j] for j in range(3)], [zm[j] for j in range(3)]

    nb = (rows + 1023) // 1024
    roots = torch.zeros((3, N, nb), dtype=torch.int32, device="cuda")
    ref = torch.zeros((3, Q), dtype=torch.uint8, device="cuda")
    ipc.ipc_compare(zcs, zms, ldz, N, rows, 0, tags, SEEDS, THR_A, 5, roots, nb)
    ipc.ipc_or_finalize(roots, nb, nb, 5, Q, R, tags, SEEDS, ref)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    assert ((ref[0] ^ ref[1] ^ ref[2]) & 1).tolist() == [1, 0, 1]

    # two calls in a row share the fixed scratch: the first on the current stream, the second
    # on an explicit non-default stream
    side = torch.cuda.Stream()
    for st in (None, side):
        out = torch.full((3, Q), 7, dtype=torch.uint8, device="cuda")
        if st is not None:
            st.wait_stream(torch.cuda.current_stream())
        ipc.ipc_compare_or_noalloc(zcs, zms, ldz, Q, R, rows, tags, SEEDS, THR_A, out, stream=st)
        torch.cuda.synchronize()
        ipc.ipc_status()
        assert (out.cpu().numpy() == ref).all()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_04463_gb300 as ipc
    z = torch.zeros(16, dtype=torch.int16, device="cuda")
    tags = torch.zeros(2, dtype=torch.int32, device="cuda")
    out = torch.zeros(3 * 256, dtype=torch.uint8, device="cuda")
    # 3 * 256 * 31 * ceil(1e6 / 1024) words > 2^20: refused before any launch
    with pytest.raises(ipc.IpcError) as e:
        ipc.ipc_compare_or_noalloc([z] * 3, [z] * 3, 1_000_000, 256, 31, 1_000_000, tags, SEEDS, THR_A, out)
    assert e.value.rc == ipc.IPC_EINVAL
    assert "exceed the fixed scratch" in ipc.ipc_last_error()
