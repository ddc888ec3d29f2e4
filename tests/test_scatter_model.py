"""Host-side model of the redistribution's write positions (no GPU): the
counters are laid out bucket-major per segment, (bucket, tile) in that order,
and one exclusive scan over them gives each tile's start in each bucket;
inside a tile a warp's elements follow the warps before it, and inside a warp
the elements follow its earlier steps and its lower lanes.  The model checks
the properties the kernels rely on: the counts sum to n, every bucket's
positions form one contiguous range in bucket order, no two elements get the
same position, and the order inside a bucket is the input order (stable) --
the same permutation as a stable sort by bucket."""
import numpy as np
import pytest

TILE, WARPS, LANES = 4096, 8, 32
SPAN = TILE // WARPS          # contiguous elements per warp
STEPS = SPAN // LANES         # elements per lane


def _positions(bucket, B):
    """Write position of every element of one segment, computed the way the
    kernels assign them (counts, bucket-major scan, warp offsets, lane ranks)."""
    n = bucket.shape[0]
    tiles = (n + TILE - 1) // TILE
    counts = np.zeros((B, tiles), np.int64)            # bucket-major: index b * tiles + t
    for t in range(tiles):
        counts[:, t] = np.bincount(bucket[t * TILE:(t + 1) * TILE], minlength=B)
    assert counts.sum() == n
    scan = np.concatenate([[0], np.cumsum(counts.reshape(-1))[:-1]]).reshape(B, tiles)
    pos = np.full(n, -1, np.int64)
    for t in range(tiles):
        wpos = np.zeros((WARPS, B), np.int64)          # per warp: its count, then its offset in the tile's part
        for w in range(WARPS):
            seg = bucket[t * TILE + w * SPAN: t * TILE + (w + 1) * SPAN]
            wpos[w] = np.bincount(seg, minlength=B)
        wpos = np.cumsum(wpos, axis=0) - wpos          # exclusive over warps, per bucket
        for w in range(WARPS):
            run = wpos[w].copy()                       # running offset of this warp in each bucket
            for u in range(STEPS):                     # one warp step: 32 consecutive elements
                base = t * TILE + w * SPAN + u * LANES
                lanes = bucket[base: base + LANES]
                for lane, b in enumerate(lanes):
                    rank = int(np.sum(lanes[:lane] == b))   # lower lanes with the same bucket
                    pos[base + lane] = scan[b, t] + run[b] + rank
                np.add.at(run, lanes, 1)
    return pos


@pytest.mark.parametrize("n,B,skew", [(1, 3, 0.0), (4095, 7, 0.0), (4096, 15, 0.5), (4097, 31, 0.0),
                                      (3 * 4096 + 123, 63, 0.9), (2 * 4096, 2047, 0.0)])
def test_write_positions_are_a_stable_permutation(n, B, skew):
    rng = np.random.default_rng(n + B)
    bucket = rng.integers(0, B, n)
    if skew:   # a few buckets hold most elements (equal keys, skewed inputs)
        hot = rng.random(n) < skew
        bucket[hot] = rng.integers(0, 3, int(hot.sum()))
    pos = _positions(bucket, B)
    assert sorted(pos.tolist()) == list(range(n))                       # no gaps, no overlaps
    assert np.array_equal(np.argsort(pos), np.argsort(bucket, kind="stable"))
