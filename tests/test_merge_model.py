"""Host-side model of the merge's grouped cut search (no GPU): a group of G
lanes tests G evenly spaced candidates of [lo, hi) per round and keeps the gap
between the last candidate that fails and the first that passes.  For every
monotone test it must return the first passing candidate (hi if none), like
a binary search, within about log_(G+1) of the range's length rounds."""
import math

import numpy as np
import pytest


def grouped_search(lo, hi, passes, G):
    rounds = 0
    while lo < hi:
        n = hi - lo
        probe = [lo + ((k + 1) * n) // (G + 1) for k in range(G)]
        votes = [passes(x) for x in probe]
        first = next((k for k, v in enumerate(votes) if v), G)
        nlo = probe[first - 1] + 1 if first > 0 else lo
        nhi = probe[first] if first < G else hi
        assert lo <= nlo <= nhi <= hi and (nhi - nlo) < n
        lo, hi = nlo, nhi
        rounds += 1
    return lo, rounds


@pytest.mark.parametrize("G", [1, 2, 4, 8, 16, 32])
def test_grouped_search_finds_first_passing_candidate(G):
    rng = np.random.default_rng(G)
    for _ in range(400):
        lo = int(rng.integers(0, 50))
        n = int(rng.choice([0, 1, 2, 3, 7, 8, 9, 31, 100, 1000, 2_500_000]))
        hi = lo + n
        t = int(rng.integers(lo, hi + 1))           # first passing candidate (hi: none passes)
        got, rounds = grouped_search(lo, hi, lambda x: x >= t, G)
        assert got == t
        # each round leaves at most ceil(n / (G + 1)) candidates
        bound = 0 if n == 0 else math.ceil(math.log(n + 1, G + 1)) + 1
        assert rounds <= bound, (n, G, rounds)


def test_one_lane_is_binary_search():
    """With one lane the probe is lo + n // 2, the midpoint of a binary search."""
    for n in range(1, 200):
        for t in range(0, n + 1):
            got, _ = grouped_search(0, n, lambda x: x >= t, 1)
            assert got == t
