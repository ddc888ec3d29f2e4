"""Host model of the one-pass K-way LCP merge (ss_kway.cu): sparse and dense
splitters ranked by binary search with the run order breaking ties, jobs
from one splitter's rank to the next, and per job an LCP loser tree
(Algorithm 4) whose games are LCP-Compare (Algorithm 2).

Checked against the oracle: the merged order and LCPs equal the sort of the
union, for K = 2..8 runs of random, duplicate-heavy and shared-prefix sets at
several splitter spacings; and the loser tree alone (one job over the whole
merge) stays within the theorem's bound of Delta L + n ceil(log2 K) + K
character comparisons.  This models the GPU design on the host; it is not
the oracle and shares no code with it."""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _lcp(a: bytes, b: bytes) -> int:
    n = min(len(a), len(b))
    i = 0
    while i < n and a[i] == b[i]:
        i += 1
    return i


class Counter:
    def __init__(self):
        self.chars = 0


def _cmp_from(a: bytes, b: bytes, h: int, cnt: Counter):
    """compare a and b from depth h (both share h characters): (sign, lcp),
    counting the characters compared (the deciding one, or the end)"""
    i = h
    while True:
        ca = a[i] if i < len(a) else None
        cb = b[i] if i < len(b) else None
        cnt.chars += 1
        if ca is None or cb is None or ca != cb:
            break
        i += 1
    if i >= len(a) and i >= len(b):
        return 0, i
    if i >= len(a):
        return -1, i
    if i >= len(b):
        return 1, i
    return (-1 if a[i] < b[i] else 1), i


def _place(run, r, k, s, lo, hi, h, cnt):
    """entries of run k that precede string s of run r (equal: lower run first)"""
    while lo < hi:
        mid = (lo + hi) // 2
        c, _ = _cmp_from(run[k][mid], s, h, cnt)
        before = c < 0 or (c == 0 and k < r)
        if before:
            lo = mid + 1
        else:
            hi = mid
    return lo


def _game(x, hx, y, hy, runs, cur, cnt):
    """LCP-Compare of fronts of runs x and y; (x first?, lcp of loser with winner)"""
    ex = cur[x] < len(runs[x]) if x < len(runs) else False
    ey = cur[y] < len(runs[y]) if y < len(runs) else False
    if not ey:
        return True, hy
    if not ex:
        return False, hx
    if hx > hy:
        return True, hy
    if hx < hy:
        return False, hx
    c, l = _cmp_from(runs[x][cur[x]], runs[y][cur[y]], hx, cnt)
    return (c < 0 or (c == 0 and x < y)), l


def _merge_job(runs, lcps, start, nout, first_lcp, cnt):
    """one job: outputs from the places `start` in every run, nout of them"""
    R = len(runs)
    KP = 1
    while KP < R:
        KP *= 2
    cur = list(start) + [0] * (KP - R)
    h = [0] * KP
    lose = [0] * KP
    win = [0] * (2 * KP)
    for k in range(KP):
        win[KP + k] = k
    for i in range(KP - 1, 0, -1):
        a, b = win[2 * i], win[2 * i + 1]
        a_first, hl = _game(a, h[a], b, h[b], runs, cur, cnt)
        w, l = (a, b) if a_first else (b, a)
        win[i], lose[i] = w, l
        h[l] = hl
    w = win[1]
    out = []
    for o in range(nout):
        s = runs[w][cur[w]]
        out.append((w, cur[w], first_lcp if o == 0 else h[w]))
        cur[w] += 1
        h[w] = lcps[w][cur[w]] if cur[w] < len(runs[w]) else 0
        x = w
        i = (KP + w) // 2
        while i >= 1:
            y = lose[i]
            x_first, hl = _game(x, h[x], y, h[y], runs, cur, cnt)
            if not x_first:
                lose[i], h[x], x = x, hl, y
            else:
                h[y] = hl
            i //= 2
        w = x
        del s
    return out


def kway_model(strings, cuts, sparse, dense, cnt=None):
    """merge the sorted runs strings[cuts[k]:cuts[k+1]] (each run sorted, ties
    by index); returns (perm, lcp) of the union with the run order on ties"""
    cnt = cnt or Counter()
    R = len(cuts) - 1
    runs, lcps, idx = [], [], []
    for k in range(R):
        part = list(range(cuts[k], cuts[k + 1]))
        part.sort(key=lambda i: (strings[i], i))
        runs.append([strings[i] for i in part])
        idx.append(part)
        lcps.append([0] + [_lcp(runs[k][j - 1], runs[k][j]) for j in range(1, len(part))])
    total = sum(len(r) for r in runs)
    # sparse splitters: places over whole runs, and the LCP with the next one
    spos, splcp = {}, {}
    for r in range(R):
        for i in range(0, len(runs[r]), sparse):
            s = runs[r][i]
            spos[(r, i)] = [i if k == r else _place(runs, r, k, s, 0, len(runs[k]), 0, cnt) for k in range(R)]
            j = i + sparse
            splcp[(r, i)] = min(lcps[r][i + 1:j + 1]) if j < len(runs[r]) else 0
    # dense splitters inside the brackets of the sparse ones
    jobs = []
    for r in range(R):
        for i in range(0, len(runs[r]), dense):
            sa = (i // sparse) * sparse
            s = runs[r][i]
            pos = []
            for k in range(R):
                if k == r:
                    pos.append(i)
                elif i == sa:
                    pos.append(spos[(r, sa)][k])
                else:
                    last = sa + sparse >= len(runs[r])
                    lo = spos[(r, sa)][k]
                    hi = len(runs[k]) if last else spos[(r, sa + sparse)][k]
                    hh = 0 if last else splcp[(r, sa)]
                    pos.append(_place(runs, r, k, s, lo, hi, hh, cnt))
            jobs.append((sum(pos), r, i, pos))
    ranks = sorted(j[0] for j in jobs)
    assert len(set(ranks)) == len(ranks) and ranks[0] == 0
    nxt = {g: (ranks[t + 1] if t + 1 < len(ranks) else total) for t, g in enumerate(ranks)}
    perm = [None] * total
    lcp = [None] * total
    for g, r, i, pos in jobs:
        first = 0
        if g > 0:
            first = max(lcps[k][pos[k]] if k == r else _lcp(runs[k][pos[k] - 1], runs[r][i])
                        for k in range(R) if pos[k] > 0)
        for o, (w, e, l) in enumerate(_merge_job(runs, lcps, pos, nxt[g] - g, first, cnt)):
            perm[g + o] = idx[w][e]
            lcp[g + o] = l
    return np.array(perm, np.uint32), np.array(lcp, np.uint32)


def _strings(ss):
    return [ss.string(i) for i in range(ss.n)]


CASES = [
    (lambda: W.random_lower(3000, seed=81), "random"),
    (lambda: W.url_like(3000, seed=82), "url"),
    (lambda: W.from_bytes_list([b"ab"[i % 2: i % 2 + 1] * (i % 5) for i in range(1500)]), "duplicates"),
    (lambda: W.dna_windows(2000, 4000, 30, seed=83), "dna"),
]


@pytest.mark.parametrize("make,name", CASES)
@pytest.mark.parametrize("K,sparse,dense", [(2, 64, 8), (4, 256, 16), (5, 32, 4), (8, 128, 128)])
def test_kway_model_equals_the_oracle(make, name, K, sparse, dense):
    ss = make()
    strs = _strings(ss)
    rng = np.random.default_rng(K * 7 + len(name))
    cuts = [0] + sorted(rng.integers(1, ss.n, K - 1).tolist()) + [ss.n]
    cuts = sorted(set(cuts))
    perm, lcp = kway_model(strs, cuts, sparse, dense)
    want_perm, want_lcp = oracle.sort(ss)
    assert np.array_equal(perm, want_perm), name
    assert np.array_equal(lcp, want_lcp), name


@pytest.mark.parametrize("K", [2, 3, 4, 8])
def test_loser_tree_comparisons_within_the_theorem_bound(K):
    """one job over the whole merge: character comparisons of the tree's games
    <= Delta L + n ceil(log2 K) + K (Algorithm 4's theorem), where Delta L =
    L(merged) - sum L(runs)"""
    ss = W.url_like(2000, seed=90 + K)
    strs = _strings(ss)
    n = ss.n
    cuts = [n * k // K for k in range(K + 1)]
    runs, lcps, idx = [], [], []
    for k in range(K):
        part = sorted(range(cuts[k], cuts[k + 1]), key=lambda i: (strs[i], i))
        runs.append([strs[i] for i in part])
        idx.append(part)
        lcps.append([0] + [_lcp(runs[k][j - 1], runs[k][j]) for j in range(1, len(part))])
    cnt = Counter()
    out = _merge_job(runs, lcps, [0] * K, n, 0, cnt)
    merged = [runs[w][e] for w, e, _ in out]
    assert merged == sorted(strs)
    L_out = sum(_lcp(merged[i - 1], merged[i]) for i in range(1, n))
    dL = L_out - sum(sum(l) for l in lcps)
    assert cnt.chars <= dL + n * math.ceil(math.log2(K)) + K, (cnt.chars, dL)
    assert [l for _, _, l in out][1:] == [_lcp(merged[i - 1], merged[i]) for i in range(1, n)]
