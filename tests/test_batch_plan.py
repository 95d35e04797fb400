"""The batched sweep's work split (soma_batch_plan: host logic, no GPU).

Whatever the split, the blocks' items must cover every tile of every member
exactly once (a tile taken twice would move its particles twice in one sweep,
a tile missed would not move them).  The balanced split (item_tiles 0) must
give block j exactly the tiles [T j / grid, T (j+1) / grid) of the members'
concatenation, in order, so that the blocks' shares differ by at most one
tile; fixed-length items are runs of at most item_tiles tiles of one member.
"""
import numpy as np
import pytest

from paper_1711_03828_gb300 import SomaError, batch_plan


def _coverage(member_tiles, items):
    seen = [np.zeros(t, np.int64) for t in member_tiles]
    for m, a, b in items.tolist():
        assert a <= b <= member_tiles[m]
        seen[m][a:b] += 1
    return seen


CASES = [([5], 1), ([5], 7), ([1, 1, 1], 2), ([128, 129, 17, 17, 18, 17, 134], 456),
         ([128, 129, 17, 17, 18, 17, 134], 152), ([0, 3, 0, 4], 3), ([1000, 1, 1000], 7)]


@pytest.mark.parametrize("member_tiles,grid", CASES)
def test_balanced_split_gives_each_block_its_equal_range(member_tiles, grid):
    items = batch_plan(member_tiles, grid, 0)
    assert len(items) % grid == 0 and len(items) >= grid
    for s in _coverage(member_tiles, items):
        assert np.all(s == 1)
    begin = np.concatenate([[0], np.cumsum(member_tiles)])
    T = int(begin[-1])
    rounds = len(items) // grid
    shares = []
    for j in range(grid):
        pieces = [items[r * grid + j] for r in range(rounds)]
        pieces = [p for p in pieces if p[2] > p[1]]
        g = [(int(begin[m]) + int(a), int(begin[m]) + int(b)) for m, a, b in pieces]
        lo, hi = T * j // grid, T * (j + 1) // grid
        if g:
            assert g[0][0] == lo and g[-1][1] == hi
            for (a0, b0), (a1, b1) in zip(g, g[1:]):
                assert b0 == a1                      # contiguous, in order
        else:
            assert lo == hi
        shares.append(hi - lo)
    assert max(shares) - min(shares) <= 1


def test_balanced_split_on_random_batches():
    rng = np.random.default_rng(11)
    for _ in range(40):
        tiles = rng.integers(1, 700, rng.integers(1, 80)).tolist()
        grid = int(rng.integers(1, 1200))
        items = batch_plan(tiles, grid, 0)
        for s in _coverage(tiles, items):
            assert np.all(s == 1)
        pieces_per_block = np.zeros(grid, np.int64)
        for i, (m, a, b) in enumerate(items.tolist()):
            pieces_per_block[i % grid] += b > a
        # one piece per member that the block's range overlaps, no more
        begin = np.concatenate([[0], np.cumsum(tiles)])
        T = int(begin[-1])
        for j in range(grid):
            lo, hi = T * j // grid, T * (j + 1) // grid
            want = sum(1 for k in range(len(tiles)) if min(hi, begin[k + 1]) > max(lo, begin[k]))
            assert pieces_per_block[j] == want
        assert len(items) // grid == max(1, pieces_per_block.max())


@pytest.mark.parametrize("item_tiles", [1, 16, 64, 256])
def test_fixed_items_are_runs_of_one_member(item_tiles):
    tiles = [128, 129, 17, 1, 300]
    items = batch_plan(tiles, 456, item_tiles)
    for s in _coverage(tiles, items):
        assert np.all(s == 1)
    assert np.all(items[:, 2] - items[:, 1] <= item_tiles)
    assert np.all(items[:, 2] > items[:, 1])
    # member order, each member's runs in order
    key = items[:, 0].astype(np.int64) * 10**6 + items[:, 1]
    assert np.all(np.diff(key) > 0)
    assert len(items) == sum(-(-t // item_tiles) for t in tiles)


def test_plan_refuses_bad_arguments():
    for args in [([], 4, 0), ([3], 0, 0), ([3], 4, -1), ([3], 1 << 21, 0)]:
        with pytest.raises(SomaError):
            batch_plan(*args)
