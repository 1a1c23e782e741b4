"""Host-side logic of the serving loop (no GPU): the tile list of the active column ranges and
the first-fit slot allocator, against brute force."""
import numpy as np
import pytest

ipc = pytest.importorskip("paper_2405_04463_gb300.binding")


@pytest.mark.parametrize("tile_cols", [32, 64, 128, 256])
def test_tile_list_is_the_sorted_union_of_covered_tiles(tile_cols):
    rng = np.random.default_rng(tile_cols)
    for _ in range(200):
        k = int(rng.integers(0, 6))
        col0 = rng.integers(0, 5000, size=k)
        ncols = rng.integers(0, 800, size=k)
        expect = sorted({c // tile_cols for a, n in zip(col0, ncols) for c in range(a, a + n)})
        assert ipc.ipc_serve_tile_list(col0, ncols, tile_cols).tolist() == expect


def test_tile_list_edges():
    # a range ending exactly on a tile boundary does not touch the next tile
    assert ipc.ipc_serve_tile_list([0], [256], 256).tolist() == [0]
    assert ipc.ipc_serve_tile_list([255], [2], 256).tolist() == [0, 1]
    assert ipc.ipc_serve_tile_list([], [], 128).tolist() == []
    assert ipc.ipc_serve_tile_list([10], [0], 128).tolist() == []


def test_first_fit_matches_brute_force():
    rng = np.random.default_rng(7)
    for _ in range(500):
        n = int(rng.integers(1, 40))
        used = (rng.random(n) < rng.random()).astype(np.uint8)
        want = int(rng.integers(1, 10))
        expect = next((s for s in range(n - want + 1) if not used[s:s + want].any()), -1)
        assert ipc.ipc_serve_first_fit(used, want) == expect
