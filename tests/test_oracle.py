"""Pins for the CPU oracle (no GPU).

Each test checks the oracle against something other than itself: Python's
own byte-string ordering and ``os.path.commonprefix`` (library routines),
``bisect`` / ``numpy.argsort(kind="stable")`` for the single S5 step,
brute force over tiny inputs, closed forms and the values the paper prints
(fixtures under tests/golden/, each with its citation).
"""
import bisect
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _py_sort(strs):
    perm = sorted(range(len(strs)), key=lambda i: (strs[i], i))
    lcp = [0] * len(strs)
    for k in range(1, len(strs)):
        lcp[k] = len(os.path.commonprefix([strs[perm[k - 1]], strs[perm[k]]]))
    return perm, lcp


def _layouts(strs):
    """The same strings as NUL-terminated, explicit-length and (if equal length) fixed-length sets."""
    out = [W.from_bytes_list(strs, terminated=True), W.from_bytes_list(strs, terminated=False)]
    if strs and len({len(s) for s in strs}) == 1 and len(strs[0]) > 0:
        ss = W.from_bytes_list(strs, terminated=False)
        out.append(W.StringSet(ss.chars, ss.offsets, None, len(strs[0]), "fixed"))
    return out


# ------------------------------------------------------------------ sort

def test_sort_brute_force_small_alphabet():
    """Every multiset of up to 4 strings over {a,b} of length <= 2, every order."""
    alphabet = [b"", b"a", b"b", b"aa", b"ab", b"ba", b"bb"]
    for n in range(0, 5):
        for combo in itertools.combinations_with_replacement(alphabet, n):
            for order in set(itertools.permutations(combo)):
                strs = list(order)
                want_perm, want_lcp = _py_sort(strs)
                for ss in _layouts(strs):
                    perm, lcp = oracle.sort(ss)
                    assert perm.tolist() == want_perm, (strs, ss.name)
                    assert lcp.tolist() == want_lcp, (strs, ss.name)


def test_sort_random_against_python():
    rng = np.random.default_rng(7)
    for trial in range(30):
        n = int(rng.integers(1, 300))
        strs = [bytes(rng.integers(1, 4, int(rng.integers(0, 12))).astype(np.uint8)) for _ in range(n)]
        want_perm, want_lcp = _py_sort(strs)
        for ss in _layouts(strs):
            perm, lcp = oracle.sort(ss)
            assert perm.tolist() == want_perm
            assert lcp.tolist() == want_lcp


def test_sort_high_bytes_are_unsigned():
    strs = [b"\xff", b"\x01", b"\x80\x01", b"\x7f\xff", b"\x80"]
    want_perm, want_lcp = _py_sort(strs)
    for ss in _layouts(strs):
        perm, lcp = oracle.sort(ss)
        assert perm.tolist() == want_perm == [1, 3, 4, 2, 0]
        assert lcp.tolist() == want_lcp


def test_pseudocode_example():
    """Section 2.1's array A = [(i^2 mod 7, i) | i in [0:5)] sorted as 2-character strings."""
    lines = [l.split() for l in open(os.path.join(GOLDEN, "pseudocode_example.txt")) if l.strip() and not l.startswith("#")]
    pairs = [tuple(int(v) for v in l) for l in lines[:5]]
    assert pairs == [((i * i) % 7, i) for i in range(5)]
    strs = [bytes([a + 1, b + 1]) for a, b in pairs]
    perm, lcp = oracle.sort(W.from_bytes_list(strs))
    assert perm.tolist() == [int(v) for v in lines[5]]
    assert lcp.tolist() == [int(v) for v in lines[6]]


def test_sort_fixed_windows_of_one_text():
    """Overlapping fixed-length windows of one text (the DNA layout)."""
    ss = W.dna_windows(n=2000, text_len=3000, window=20, seed=9)
    strs = [ss.string(i) for i in range(ss.n)]
    assert all(len(s) == 20 for s in strs)
    want_perm, want_lcp = _py_sort(strs)
    perm, lcp = oracle.sort(ss)
    assert perm.tolist() == want_perm
    assert lcp.tolist() == want_lcp


# ------------------------------------------------------------- D and L

def _brute_D(strs):
    """D by definition: for each string the shortest prefix (terminator counted as a
    character) that is no prefix of any other string's terminated form."""
    ts = [s + b"\0" for s in strs]
    D = 0
    for i, s in enumerate(ts):
        k = 1
        while k < len(s) and any(j != i and t[:k] == s[:k] for j, t in enumerate(ts)):
            k += 1
        D += k
    return D


def test_D_L_brute_force():
    rng = np.random.default_rng(3)
    for trial in range(200):
        n = int(rng.integers(1, 12))
        strs = [bytes(rng.integers(1, 3, int(rng.integers(0, 5))).astype(np.uint8)) for _ in range(n)]
        ss = W.from_bytes_list(strs)
        perm, lcp = oracle.sort(ss)
        L, D, N = oracle.stats(ss, perm, lcp)
        assert L == sum(lcp.tolist())
        assert D == _brute_D(strs)
        assert N == sum(len(s) + 1 for s in strs)
        assert L + n <= D <= 2 * L + n


def test_D_L_bounds_url_sample():
    ss = W.url_like(n=20000, seed=2)
    perm, lcp = oracle.sort(ss)
    L, D, N = oracle.stats(ss, perm, lcp)
    assert L + ss.n <= D <= 2 * L + ss.n
    assert D <= N


@pytest.mark.slow
def test_table3_sinha_dna_statistics():
    """Table 3: length-9 DNA strings, n = 31.6 M: D/N = 100.0 %, L/n = 9.0."""
    row = [l.split() for l in open(os.path.join(GOLDEN, "table3_sinha_dna.txt")) if l.strip() and not l.startswith("#")][0]
    n, length, sigma = int(row[0]), int(row[1]), int(row[2])
    dn, ln = float(row[3]), float(row[4])
    assert sigma == 4
    ss = W.sinha_dna_like(n, length=length)
    perm, lcp = oracle.sort(ss)
    L, D, N = oracle.stats(ss, perm, lcp)
    assert N == n * (length + 1)
    assert round(100.0 * D / N, 1) == dn
    assert round(L / n, 1) == ln


# ----------------------------------------------------------- chars_h

def test_chars_h_literals():
    ss = W.from_bytes_list([b"abcdefghij", b"ab", b""])
    assert oracle.chars_h(ss, 0, 0) == 0x6162636465666768
    assert oracle.chars_h(ss, 0, 3) == 0x6465666768696A00
    assert oracle.chars_h(ss, 1, 0) == 0x6162000000000000
    assert oracle.chars_h(ss, 1, 2) == 0
    assert oracle.chars_h(ss, 2, 0) == 0


def test_chars_h_against_bytes():
    rng = np.random.default_rng(5)
    strs = [bytes(rng.integers(1, 256, int(rng.integers(0, 30))).astype(np.uint8)) for _ in range(200)]
    for ss in _layouts(strs):
        depth = rng.integers(0, 32, len(strs)).astype(np.uint64)
        keys = oracle.chars_h_all(ss, depth)
        for i, s in enumerate(strs):
            h = int(depth[i])
            assert int(keys[i]) == int.from_bytes(s[h:h + 8].ljust(8, b"\0"), "big")


# ---------------------------------------------------- one S5 step (Alg. 1)

def test_fig1_tree_level_order():
    lines = [l.split() for l in open(os.path.join(GOLDEN, "fig1_tree_v7.txt")) if l.strip() and not l.startswith("#")]
    level_order = [int(v) for v in lines[0]]
    x = np.array([10 * (i + 1) for i in range(7)], np.uint64)
    t = oracle.s5_tree(x)
    assert t.tolist() == [int(x[i]) for i in level_order]
    # equality buckets of Figure 1
    eq = [int(v) for v in lines[1]]
    b = oracle.s5_classify(x, x)
    assert b.tolist() == eq


def _closed_form_bucket(c, x):
    r = bisect.bisect_left(list(x), c)
    return 2 * r + (1 if r < len(x) and x[r] == c else 0)


@pytest.mark.parametrize("d", [1, 2, 3, 5, 8, 10])
def test_s5_classify_closed_form(d):
    rng = np.random.default_rng(d)
    v = (1 << d) - 1
    x = np.sort(rng.integers(0, 4 * v + 8, v).astype(np.uint64))   # duplicates allowed
    keys = rng.integers(0, 4 * v + 10, 5000).astype(np.uint64)
    keys[:v] = x
    b = oracle.s5_classify(keys, x)
    want = [_closed_form_bucket(int(c), [int(y) for y in x]) for c in keys]
    assert b.tolist() == want


def test_s5_classify_full_64bit_keys():
    rng = np.random.default_rng(11)
    v = 255
    x = np.sort(rng.integers(0, 2**64, v, dtype=np.uint64))
    keys = np.concatenate([rng.integers(0, 2**64, 3000, dtype=np.uint64), x,
                           np.array([0, 2**64 - 1], np.uint64)])
    b = oracle.s5_classify(keys, x)
    xs = [int(y) for y in x]
    assert b.tolist() == [_closed_form_bucket(int(c), xs) for c in keys]


def test_fig1_s5_equal():
    """S5-Equal on Figure 1's tree: each splitter lands in its equality bucket
    (stopping at its own node, whichever level), keys between splitters in the
    even buckets."""
    lines = [l.split() for l in open(os.path.join(GOLDEN, "fig1_tree_v7.txt")) if l.strip() and not l.startswith("#")]
    eq = [int(v) for v in lines[1]]
    x = np.array([10 * (i + 1) for i in range(7)], np.uint64)
    assert oracle.s5_classify_equal(x, x).tolist() == eq
    between = np.array([5 + 10 * i for i in range(8)], np.uint64)   # below x0, between, above x6
    assert oracle.s5_classify_equal(between, x).tolist() == [2 * i for i in range(8)]


@pytest.mark.parametrize("d", [1, 2, 3, 4, 6, 8, 10])
def test_s5_equal_distinct_splitters_closed_form(d):
    """With distinct splitters S5-Equal gives the closed-form bucket."""
    rng = np.random.default_rng(100 + d)
    v = (1 << d) - 1
    x = np.sort(rng.choice(10 * v + 20, v, replace=False).astype(np.uint64) + 1)
    keys = np.concatenate([rng.integers(0, 10 * v + 30, 4000).astype(np.uint64), x, x - 1, x + 1])
    xs = [int(y) for y in x]
    assert oracle.s5_classify_equal(keys, x).tolist() == [_closed_form_bucket(int(c), xs) for c in keys]


def _highest_copy(xs, c):
    """Among the in-order positions k with x_k = c (a contiguous range), the one
    highest in the complete tree: the most trailing zero bits of k + 1."""
    ks = [k for k, y in enumerate(xs) if y == c]
    return max(ks, key=lambda k: ((k + 1) & -(k + 1)))


@pytest.mark.parametrize("d", [1, 2, 3, 5, 7, 9])
def test_s5_equal_repeated_splitters(d):
    """Repeated splitter values (what the pick emits for a sample with few
    distinct keys): keys equal to no splitter keep the closed-form bucket; a
    key equal to a splitter value lands in the equality bucket of the copy
    highest in the tree; distributing by either bucketing gives the same
    order."""
    rng = np.random.default_rng(200 + d)
    v = (1 << d) - 1
    x = np.sort(rng.integers(0, max(3, v // 3), v).astype(np.uint64) * 4)   # many repeats
    keys = rng.integers(0, 4 * max(3, v // 3) + 4, 3000).astype(np.uint64)
    xs = [int(y) for y in x]
    b_eq = oracle.s5_classify_equal(keys, x)
    b_cf = oracle.s5_classify(keys, x)
    for c, be, bc in zip(keys.tolist(), b_eq.tolist(), b_cf.tolist()):
        if c in xs:
            assert be == 2 * _highest_copy(xs, c) + 1
        else:
            assert be == bc
    assert np.argsort(b_eq, kind="stable").tolist() == np.argsort(b_cf, kind="stable").tolist()


def test_s5_distribute_stable():
    rng = np.random.default_rng(2)
    v = 31
    bucket = rng.integers(0, 2 * v + 1, 10000).astype(np.uint16)
    bb, out = oracle.s5_distribute(bucket, v)
    counts = np.bincount(bucket, minlength=2 * v + 1)
    assert bb.tolist() == [0] + np.cumsum(counts).tolist()
    assert out.tolist() == np.argsort(bucket, kind="stable").tolist()


def test_s5_pick_distinct_sample_is_equidistant():
    """With distinct samples of size alpha*v + alpha - 1 (alpha = 2), the recursive
    scheme picks the equidistant splitters p_alpha, p_2alpha, ... of Algorithm 1."""
    rng = np.random.default_rng(4)
    for d in range(1, 11):
        v = (1 << d) - 1
        a = 2 * v + 1
        sample = np.sort(rng.choice(10**9, a, replace=False).astype(np.uint64))
        x = oracle.s5_pick(sample, v)
        assert x.tolist() == [int(sample[2 * (i + 1) - 1]) for i in range(v)]


def test_s5_pick_duplicates_sorted_subset():
    rng = np.random.default_rng(6)
    for trial in range(50):
        d = int(rng.integers(1, 9))
        v = (1 << d) - 1
        a = 2 * v + 1
        sample = np.sort(rng.integers(0, int(rng.integers(1, 40)), a).astype(np.uint64))
        x = oracle.s5_pick(sample, v)
        assert np.all(np.diff(x.astype(np.int64)) >= 0)
        assert set(x.tolist()) <= set(sample.tolist())
        # the root of the tree is the middle sample
        assert int(x[v // 2]) == int(sample[a // 2])
        # equal samples are skipped: a value appears as a splitter in one run only
        vals = x.tolist()
        runs = [k for k, _ in itertools.groupby(vals)]
        assert len(runs) == len(set(vals))
    same = np.full(15, 42, np.uint64)
    assert oracle.s5_pick(same, 7).tolist() == [42] * 7


# ------------------------------------------ LCP insertion sort (Alg. 5)

def test_lcp_insertion_sort_matches_and_bound():
    rng = np.random.default_rng(8)
    for trial in range(60):
        n = int(rng.integers(1, 80))
        strs = [bytes(rng.integers(1, 3, int(rng.integers(0, 10))).astype(np.uint8)) for _ in range(n)]
        ss = W.from_bytes_list(strs)
        want_perm, want_lcp = _py_sort(strs)
        s, h, ncmp = oracle.lcp_insertion(ss, np.arange(n))
        assert s.tolist() == want_perm
        assert h.tolist() == want_lcp
        assert ncmp <= sum(want_lcp) + n * (n - 1) // 2


def test_lcp_insertion_sort_common_prefix():
    rng = np.random.default_rng(9)
    pre = b"common/"
    strs = [pre + bytes(rng.integers(1, 4, int(rng.integers(0, 6))).astype(np.uint8)) for _ in range(50)]
    ss = W.from_bytes_list(strs)
    s, h, _ = oracle.lcp_insertion(ss, np.arange(50), hbar=len(pre))
    want_perm, want_lcp = _py_sort(strs)
    assert s.tolist() == want_perm
    assert h.tolist()[1:] == want_lcp[1:]


# -------------------------------------------------- LCP-Compare (Alg. 2)

def test_lcp_compare_cases():
    rng = np.random.default_rng(10)
    for trial in range(500):
        strs = sorted(bytes(rng.integers(1, 3, int(rng.integers(0, 7))).astype(np.uint8)) for _ in range(3))
        p = strs[0]
        a, b = strs[1], strs[2]
        if rng.random() < 0.5:
            a, b = b, a
        ss = W.from_bytes_list([p, a, b])
        ha = len(os.path.commonprefix([p, a]))
        hb = len(os.path.commonprefix([p, b]))
        (x, hx, y, hp), _ = oracle.lcp_compare(ss, 1, ha, 2, hb)
        small = 1 if (a, 1) <= (b, 2) else 2
        assert x == small and y == 3 - small
        assert hx == (ha if small == 1 else hb)
        assert hp == len(os.path.commonprefix([a, b]))


# ------------------------------------------------ LCP merges (Alg. 3, 4)

def _runs(ss, K, rng):
    """Split the index range into K contiguous chunks, sort each with the oracle."""
    cuts = np.sort(rng.integers(0, ss.n + 1, K - 1))
    begin = np.concatenate([[0], cuts, [ss.n]]).astype(np.uint64)
    s_parts, h_parts = [], []
    for k in range(K):
        b, e = int(begin[k]), int(begin[k + 1])
        sub = W.subset(ss, np.arange(b, e))
        p, h = oracle.sort(sub)
        s_parts.append((p + b).astype(np.uint32))
        h_parts.append(h)
    return begin, np.concatenate(s_parts) if s_parts else np.zeros(0, np.uint32), np.concatenate(h_parts)


@pytest.mark.parametrize("gen", ["url", "dup", "lower"])
def test_lcp_merge2(gen):
    rng = np.random.default_rng(12)
    ss = {"url": lambda: W.url_like(3000, seed=21),
          "dup": lambda: W.from_bytes_list([bytes(rng.integers(1, 3, int(rng.integers(0, 6))).astype(np.uint8)) for _ in range(800)]),
          "lower": lambda: W.random_lower(3000, seed=22, min_len=1, max_len=6)}[gen]()
    for trial in range(5):
        begin, s, h = _runs(ss, 2, rng)
        m = int(begin[1])
        out, hout, ncmp = oracle.lcp_merge2(ss, s[:m], h[:m], s[m:], h[m:])
        perm, lcp = oracle.sort(ss)
        assert out.tolist() == perm.tolist()
        assert hout.tolist() == lcp.tolist()
        dL = int(lcp.astype(np.int64).sum() - h[:m].astype(np.int64)[1:].sum() - h[m:].astype(np.int64)[1:].sum())
        assert ncmp <= dL + ss.n


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5, 8, 13])
def test_lcp_mergek(K):
    rng = np.random.default_rng(100 + K)
    for ss in (W.url_like(2000, seed=23),
               W.from_bytes_list([bytes(rng.integers(1, 3, int(rng.integers(0, 6))).astype(np.uint8)) for _ in range(600)])):
        begin, s, h = _runs(ss, K, rng)
        out, hout, ncmp = oracle.lcp_mergek(ss, s, h, begin)
        perm, lcp = oracle.sort(ss)
        assert out.tolist() == perm.tolist()
        assert hout.tolist() == lcp.tolist()
        sumL_runs = sum(int(h[int(begin[k]) + 1:int(begin[k + 1])].astype(np.int64).sum()) for k in range(K))
        dL = int(lcp.astype(np.int64).sum()) - sumL_runs
        Kp = 1 << max(0, math.ceil(math.log2(K))) if K > 1 else 1
        assert ncmp <= dL + ss.n * math.log2(Kp) + Kp


# ------------------------------------------------ the any-size checker

def test_check_sorted_accepts_oracle_output_and_catches_planted_mistakes():
    ss = W.url_like(30000, seed=41)
    perm, lcp = oracle.sort(ss)
    assert oracle.check_sorted(ss, perm, lcp) == (0, ss.n)
    rng = np.random.default_rng(1)
    for _ in range(20):
        p2, l2 = perm.copy(), lcp.copy()
        kind = rng.integers(0, 4)
        i = int(rng.integers(1, ss.n - 1))
        if kind == 0:     # swap two neighbours
            p2[i], p2[i + 1] = p2[i + 1], p2[i]
        elif kind == 1:   # an LCP off by one
            l2[i] += 1
        elif kind == 2:   # a duplicated index (not a permutation)
            p2[i] = p2[i - 1]
        else:             # nonzero first LCP
            l2[0] = 1
        bad, first = oracle.check_sorted(ss, p2, l2)
        assert bad > 0 and first <= max(i + 1, 1)


def test_check_sorted_tie_order():
    ss = W.from_bytes_list([b"x", b"x", b"a"])
    assert oracle.check_sorted(ss, np.array([2, 0, 1]), np.array([0, 0, 1])) == (0, 3)
    assert oracle.check_sorted(ss, np.array([2, 1, 0]), np.array([0, 0, 1]))[0] == 1   # equal strings out of index order


# ------------------------------------------- parallel library-sort baseline

def test_parallel_baseline_equals_oracle():
    """The CPU baseline that sorts with a parallel library stable sort gives
    the oracle's perm and lcp (same order, ties by index) on every layout."""
    sets = [W.random_lower(30_000, seed=31, min_len=0, max_len=12), W.url_like(20_000, seed=32),
            W.sinha_dna_like(20_000, seed=33), W.dna_windows(15_000, 300_100, 100, seed=34),
            W.paper_random(20_000, seed=35),
            W.from_bytes_list([b"ab", b"", b"a", b"ab", b"b\xff", b"b", b""] * 300, terminated=False)]
    for ss in sets:
        want_perm, want_lcp = oracle.sort(ss)
        perm, lcp, used = oracle.sort_parallel(ss, threads=4)
        assert used >= 1
        assert np.array_equal(perm, want_perm), ss.name
        assert np.array_equal(lcp, want_lcp), ss.name
