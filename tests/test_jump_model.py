"""Host-side model of the jump-table classifier (no GPU): the table covers
the 10 key bits after the prefix all splitters share; keys outside that
prefix go straight to the outer buckets; an entry holds the first node whose
splitter lies inside its key range (or the leaf all its keys reach); the
descent finishes from there and tests equality once.  Every bucket must be
the closed form 2r + [x_r = c], r = #{j : x_j < c}."""
import bisect

import numpy as np
import pytest

A = 10                       # table bits
M64 = (1 << 64) - 1


def level_order(x, d):
    t = [0] * (1 << d)
    for i in range(1, 1 << d):
        l = i.bit_length() - 1
        t[i] = x[((2 * (i - (1 << l)) + 1) << (d - l - 1)) - 1]
    return t


def jump_classify(keys, x):
    v = len(x)
    d = (v + 1).bit_length() - 1
    t = level_order(x, d)
    s = 64 if x[0] == x[-1] else 64 - (x[0] ^ x[-1]).bit_length()
    s = min(s, 64 - A)
    mask = ((M64 << (64 - s)) & M64) if s else 0
    pre = x[0] & mask
    low = 64 - s - A
    table = []
    for p in range(1 << A):
        lo = pre | (p << low)
        hi = lo | ((1 << low) - 1)
        i = 1
        while i <= v:
            if t[i] < lo:
                i = 2 * i + 1
            elif t[i] >= hi:
                i = 2 * i
            else:
                break
        table.append(i)
    out = []
    for c in keys:
        cp = c & mask
        node = v + 1 if cp < pre else 2 * v + 1 if cp > pre else table[((c << s) & M64) >> (64 - A)]
        while node <= v:
            node = 2 * node + (1 if c > t[node] else 0)
        r = node - (v + 1)
        out.append(2 * r + (1 if r < v and x[r] == c else 0))
    return out


def closed_form(keys, x):
    out = []
    for c in keys:
        r = bisect.bisect_left(x, c)
        out.append(2 * r + (1 if r < len(x) and x[r] == c else 0))
    return out


@pytest.mark.parametrize("d", [1, 2, 3, 5, 8, 10])
def test_jump_table_gives_the_closed_form(d):
    rng = np.random.default_rng(300 + d)
    v = (1 << d) - 1
    cases = []
    x = sorted(int(y) for y in rng.integers(0, 1 << 64, v, dtype=np.uint64))           # spread over 64 bits
    cases.append(x)
    pre = int.from_bytes(b"http://w", "big") & ~0xFFFFFF
    cases.append(sorted(pre | int(y) for y in rng.integers(0, 1 << 24, v)))            # 40 shared bits
    cases.append(sorted(int(y) * 8 for y in rng.integers(0, max(2, v // 3), v)))       # repeats, small values
    cases.append([12345] * v)                                                          # all equal
    for x in cases:
        keys = [int(y) for y in rng.integers(0, 1 << 64, 300, dtype=np.uint64)]
        keys += [(x[0] & ~0xFFFFFFFF) | int(y) for y in rng.integers(0, 1 << 32, 300)]
        keys += x + [(y - 1) & M64 for y in x] + [(y + 1) & M64 for y in x] + [0, M64]
        assert jump_classify(keys, x) == closed_form(keys, x)
