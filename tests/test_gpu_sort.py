"""GPU parity: the CUDA path through the C ABI against the CPU oracle,
element by element (integer outputs: bit-exact)."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import gpu_sort, to_device

pytestmark = pytest.mark.gpu


def _check(ss):
    perm, lcp = gpu_sort(ss)
    want_perm, want_lcp = oracle.sort(ss)
    if not np.array_equal(perm, want_perm):
        bad = np.flatnonzero(perm != want_perm)
        raise AssertionError(f"{ss.name}: perm differs at {bad[:10]} (of {bad.size}); got {perm[bad[:5]]} want {want_perm[bad[:5]]}")
    if not np.array_equal(lcp, want_lcp):
        bad = np.flatnonzero(lcp != want_lcp)
        raise AssertionError(f"{ss.name}: lcp differs at {bad[:10]} (of {bad.size}); got {lcp[bad[:5]]} want {want_lcp[bad[:5]]}")
    return perm, lcp


# ------------------------------------------------------------- workloads

def test_plain_random_lower_200k():
    """Plain single sort: n = 200,000, length U[8,32] over 'a'..'z', seed 1."""
    _check(W.random_lower(200_000, seed=1))


def test_url_like_small():
    _check(W.url_like(300_000, seed=2))


def test_dna_windows_small():
    _check(W.dna_windows(n=300_000, text_len=6_000_000, window=100, seed=3))


def test_no_lcp_small():
    _check(W.no_lcp(n=300_000, seed=5))


def test_paper_random_with_empty_strings():
    _check(W.paper_random(200_000, seed=11))


def test_sinha_dna_like_duplicates():
    _check(W.sinha_dna_like(400_000, seed=12))


# ------------------------------------------------------------- edge cases

def test_empty_and_single():
    import torch
    import paper_1403_2056_gb300 as P
    ss = W.from_bytes_list([b"abc"])
    perm, lcp = gpu_sort(ss)
    assert perm.tolist() == [0] and lcp.tolist() == [0]
    chars, offsets, _ = to_device(W.from_bytes_list([b"x"]))
    out = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    P.ss_sort(chars, offsets, 0, out, out)   # n = 0: no-op


@pytest.mark.parametrize("n", [2, 3, 31, 32, 33, 255, 256, 257, 511, 512, 513, 1023, 1024, 1025, 2047, 2048, 2049, 4095, 4096,
                               4097, 8191, 8192, 8193, 20000])
def test_threshold_sizes(n):
    _check(W.random_lower(n, seed=n, min_len=0, max_len=12))


def test_all_equal_long_strings():
    """One big equality bucket recursing 8 characters per level."""
    s = b"q" * 200
    _check(W.from_bytes_list([s] * 10000 + [s[:-1] + b"r"] * 3 + [s[:150]] * 5))


def test_many_duplicates_tiny_alphabet():
    rng = np.random.default_rng(1)
    strs = [bytes(rng.integers(1, 3, int(rng.integers(0, 6))).astype(np.uint8)) for _ in range(50000)]
    _check(W.from_bytes_list(strs))


def test_long_common_prefix_last_char_differs():
    rng = np.random.default_rng(2)
    pre = b"p" * 997
    strs = [pre + bytes([int(c)]) + b"z" * int(rng.integers(0, 9)) for c in rng.integers(1, 256, 30000)]
    _check(W.from_bytes_list(strs))


def test_deep_recursion_two_long_prefixes():
    """Two halves with different 1,000-character prefixes: no request-wide
    shared prefix, so both big segments recurse 8 characters per level for
    about 125 levels before their strings differ."""
    rng = np.random.default_rng(5)
    strs = []
    for k in range(6000):
        pre = (b"a" if k % 2 else b"b") * 1000
        strs.append(pre + bytes(rng.integers(97, 100, int(rng.integers(0, 6))).astype(np.uint8)))
    _check(W.from_bytes_list(strs))


def test_prefix_chain_and_duplicates():
    """Every string a prefix of the next ("x", "xx", ... 3,000 x's), each twice,
    shuffled: the order is by length, ties by index, and every LCP is the
    shorter length."""
    rng = np.random.default_rng(6)
    strs = [b"x" * L for L in range(1, 3001)] * 2
    order = rng.permutation(len(strs))
    _check(W.from_bytes_list([strs[i] for i in order]))


def test_explicit_lengths_long_strings():
    """Length-delimited strings of up to 4,000 bytes over two letters, packed
    back to back without terminators."""
    rng = np.random.default_rng(7)
    strs = [bytes(rng.integers(1, 3, int(rng.integers(0, 4000))).astype(np.uint8)) for _ in range(3000)]
    strs += strs[:500]   # duplicates
    _check(W.from_bytes_list(strs, terminated=False))


def test_high_bytes_and_unaligned_offsets():
    rng = np.random.default_rng(3)
    strs = [bytes(rng.integers(1, 256, int(rng.integers(0, 40))).astype(np.uint8)) for _ in range(70000)]
    _check(W.from_bytes_list(strs))


def test_explicit_lengths():
    rng = np.random.default_rng(4)
    strs = [bytes(rng.integers(1, 5, int(rng.integers(0, 30))).astype(np.uint8)) for _ in range(60000)]
    _check(W.from_bytes_list(strs, terminated=False))


def test_fixed_windows_short_text_many_duplicates():
    _check(W.dna_windows(n=100_000, text_len=20_000, window=100, seed=8))


# ---------------------------------------------------------- other entry points

def test_batch_equals_single():
    import torch
    import paper_1403_2056_gb300 as P
    sets = [W.random_lower(5000, seed=1), W.url_like(20000, seed=2), W.dna_windows(30000, 100000, 100, seed=3),
            W.from_bytes_list([b"a"]), W.from_bytes_list([]), W.random_lower(33, seed=4),
            W.url_like(100000, seed=6), W.sinha_dna_like(3000, seed=7)]
    reqs, keep = [], []
    for ss in sets:
        chars, offsets, lengths = to_device(ss)
        n = ss.n
        perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda:0")
        lcp = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda:0")
        st = torch.full((1,), 99, dtype=torch.int32, device="cuda:0")
        reqs.append(dict(chars=chars, offsets=offsets, lengths=lengths, fixed_len=ss.fixed_len, n=n,
                         perm_out=perm, lcp_out=lcp, status_out=st))
        keep.append((ss, perm, lcp, st))
    P.ss_sort_batch(reqs)
    torch.cuda.synchronize()
    for ss, perm, lcp, st in keep:
        want_perm, want_lcp = oracle.sort(ss)
        assert int(st.item()) == 0
        assert np.array_equal(perm[:ss.n].cpu().numpy().view(np.uint32), want_perm), ss.name
        assert np.array_equal(lcp[:ss.n].cpu().numpy().view(np.uint32), want_lcp), ss.name


@pytest.mark.parametrize("runs", [1, 2, 4, 5])
def test_sort_host_buffers(runs):
    import paper_1403_2056_gb300 as P
    ss = W.url_like(100_000, seed=9)
    perm = np.empty(ss.n, np.uint32)
    lcp = np.empty(ss.n, np.uint32)
    P.ss_sort_host(ss.chars, ss.offsets, None, 0, perm, lcp, runs=runs)
    want_perm, want_lcp = oracle.sort(ss)
    assert np.array_equal(perm, want_perm)
    assert np.array_equal(lcp, want_lcp)


def test_gather_keys():
    import torch
    import paper_1403_2056_gb300 as P
    rng = np.random.default_rng(5)
    strs = [bytes(rng.integers(1, 256, int(rng.integers(0, 30))).astype(np.uint8)) for _ in range(5000)]
    for ss in (W.from_bytes_list(strs), W.from_bytes_list(strs, terminated=False),
               W.dna_windows(5000, 50000, 100, seed=1)):
        lens = ss.all_lengths()
        depth = (rng.random(ss.n) * (lens.astype(np.float64) + 1)).astype(np.uint32)
        depth = np.minimum(depth, lens.astype(np.uint32))
        chars, offsets, lengths = to_device(ss)
        d = torch.from_numpy(depth.view(np.int32)).cuda()
        keys = torch.zeros(ss.n, dtype=torch.int64, device="cuda:0")
        P.ss_gather_keys(chars, offsets, lengths, ss.fixed_len, ss.n, d, keys)
        got = keys.cpu().numpy().view(np.uint64)
        want = oracle.chars_h_all(ss, depth.astype(np.uint64))
        assert np.array_equal(got, want)


@pytest.mark.parametrize("d", [1, 2, 5, 10])
def test_splitters_match_oracle_pick(d):
    import torch
    import paper_1403_2056_gb300 as P
    rng = np.random.default_rng(d)
    v = (1 << d) - 1
    a = 2 * v + 1
    for hi in (5, 50, 10**12):
        sample = rng.integers(0, hi, a).astype(np.uint64)
        s = torch.from_numpy(sample.view(np.int64)).cuda()
        x = torch.zeros(v, dtype=torch.int64, device="cuda:0")
        P.ss_splitters(s, a, d, x)
        got = x.cpu().numpy().view(np.uint64)
        want = oracle.s5_pick(np.sort(sample), v)
        assert np.array_equal(got, want)


@pytest.mark.parametrize("d,n", [(1, 1000), (3, 9000), (7, 50000), (10, 300000), (10, 0)])
def test_classify_step_matches_oracle(d, n):
    import torch
    import paper_1403_2056_gb300 as P
    rng = np.random.default_rng(d + n)
    v = (1 << d) - 1
    x = np.sort(rng.integers(0, 8 * v + 16, v).astype(np.uint64))
    keys = rng.integers(0, 8 * v + 20, n).astype(np.uint64)
    tk = torch.from_numpy(keys.view(np.int64)).cuda() if n else torch.zeros(1, dtype=torch.int64, device="cuda:0")
    tx = torch.from_numpy(x.view(np.int64)).cuda()
    b = torch.zeros(max(n, 1), dtype=torch.int16, device="cuda:0")
    bb = torch.zeros(2 * v + 2, dtype=torch.int32, device="cuda:0")
    order = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda:0")
    P.ss_classify(tk, n, tx, d, b, bb, order)
    want_b = oracle.s5_classify(keys, x)
    want_bb, want_order = oracle.s5_distribute(want_b, v)
    assert np.array_equal(b[:n].cpu().numpy().view(np.uint16), want_b)
    assert np.array_equal(bb.cpu().numpy().view(np.uint32).astype(np.uint64), want_bb)
    assert np.array_equal(order[:n].cpu().numpy().view(np.uint32).astype(np.uint64), want_order)


def _classifier_cases():
    """(name, d, splitters, keys): small integers with repeated splitters,
    distinct full-range 64-bit values, text-like keys whose splitters share a
    long prefix (keys below, inside and above it), all splitters equal, and
    splitters at 0 and 2^64 - 1; every case holds keys equal to splitters and
    their neighbours.  n spans three tiles of 4096 and a ragged tail."""
    rng = np.random.default_rng(91)
    n = 3 * 4096 + 123
    cases = []
    for d in (1, 2, 3, 5, 7, 10):
        v = (1 << d) - 1
        x = np.sort(rng.integers(0, 4 * v + 8, v)).astype(np.uint64)
        k = rng.integers(0, 4 * v + 10, n).astype(np.uint64)
        cases.append((f"small_d{d}", d, x, k))
        x = np.unique(rng.integers(1, 2**64 - 1, v + 64, dtype=np.uint64))[:v]
        k = rng.integers(0, 2**64, n, dtype=np.uint64)
        cases.append((f"full_d{d}", d, x, k))
        pre = np.uint64(int.from_bytes(b"http://w", "big") & ~0xFFFFFF)   # 40 shared bits
        x = np.sort(pre | rng.integers(0, 1 << 24, v).astype(np.uint64))
        k = pre | rng.integers(0, 1 << 24, n).astype(np.uint64)
        k[: n // 8] = rng.integers(0, 2**64, n // 8, dtype=np.uint64)   # mostly outside the prefix
        cases.append((f"prefix_d{d}", d, x, k))
    x = np.full(7, 12345, np.uint64)
    cases.append(("all_equal_d3", 3, x, rng.integers(12340, 12350, n).astype(np.uint64)))
    x = np.array([0] + sorted(rng.integers(1, 2**64 - 1, 5, dtype=np.uint64).tolist()) + [2**64 - 1], np.uint64)
    cases.append(("extremes_d3", 3, x, np.concatenate([rng.integers(0, 2**64, n - 4, dtype=np.uint64),
                                                         np.array([0, 1, 2**64 - 2, 2**64 - 1], np.uint64)])))
    out = []
    for name, d, x, k in cases:
        k = k.copy()
        m = min(len(x), n // 4)
        k[-3 * m:] = np.concatenate([x[:m], x[:m] - np.uint64(1), x[:m] + np.uint64(1)])   # wraps at the extremes
        out.append((name, d, x, k))
    return out


@pytest.mark.parametrize("cls", [0, 1, 2])
def test_classifiers_match_oracle(cls):
    """ss_classify_ex with each classifier against the oracle: S5-Unroll and
    the jump table give the closed-form bucket (orc_s5_classify), S5-Equal the
    oracle's S5-Equal buckets; bucket starts and the stable order follow."""
    import torch
    import paper_1403_2056_gb300 as P
    for name, d, x, keys in _classifier_cases():
        n, v = keys.shape[0], (1 << d) - 1
        tk = torch.from_numpy(keys.view(np.int64)).cuda()
        tx = torch.from_numpy(x.view(np.int64)).cuda()
        b = torch.zeros(n, dtype=torch.int16, device="cuda:0")
        bb = torch.zeros(2 * v + 2, dtype=torch.int32, device="cuda:0")
        order = torch.zeros(n, dtype=torch.int32, device="cuda:0")
        P.ss_classify_ex(tk, n, tx, d, cls, b, bb, order)
        want_b = oracle.s5_classify_equal(keys, x) if cls == 1 else oracle.s5_classify(keys, x)
        want_bb, want_order = oracle.s5_distribute(want_b, v)
        assert np.array_equal(b.cpu().numpy().view(np.uint16), want_b), (name, cls)
        assert np.array_equal(bb.cpu().numpy().view(np.uint32).astype(np.uint64), want_bb), (name, cls)
        assert np.array_equal(order.cpu().numpy().view(np.uint32).astype(np.uint64), want_order), (name, cls)


def test_mixed_classifiers_in_one_batch():
    """Requests with different classifiers in one batch (jump tables built for
    the jump requests' segments only): each result is the oracle's."""
    import torch
    import paper_1403_2056_gb300 as P
    sets = [W.url_like(80_000, seed=51), W.sinha_dna_like(70_000, seed=52), W.random_lower(90_000, seed=53),
            W.dna_windows(60_000, 1_200_100, 100, seed=54), W.paper_random(50_000, seed=55), W.url_like(9_000, seed=56)]
    reqs, outs = [], []
    for ss in sets:
        chars, offsets, lengths = to_device(ss)
        perm = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
        lcp = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
        reqs.append(dict(chars=chars, offsets=offsets, lengths=lengths, fixed_len=ss.fixed_len, n=ss.n,
                         perm_out=perm, lcp_out=lcp))
        outs.append((perm, lcp))
    P.ss_sort_batch_tuned(reqs, [(0, 0, k % 3) for k in range(len(reqs))])
    torch.cuda.synchronize()
    for k, (ss, (perm, lcp)) in enumerate(zip(sets, outs)):
        want_perm, want_lcp = oracle.sort(ss)
        assert np.array_equal(perm.cpu().numpy().view(np.uint32), want_perm), (ss.name, k % 3)
        assert np.array_equal(lcp.cpu().numpy().view(np.uint32), want_lcp), (ss.name, k % 3)


@pytest.mark.parametrize("K", [1, 2, 3, 4, 7, 16])
def test_merge_runs(K):
    import torch
    import paper_1403_2056_gb300 as P
    rng = np.random.default_rng(K)
    for ss in (W.url_like(120_000, seed=K), W.sinha_dna_like(50_000, seed=K)):
        cuts = np.sort(rng.integers(0, ss.n + 1, K - 1))
        rb = np.concatenate([[0], cuts, [ss.n]]).astype(np.uint32)
        run_perm = np.empty(ss.n, np.uint32)
        run_lcp = np.empty(ss.n, np.uint32)
        for k in range(K):
            b, e = int(rb[k]), int(rb[k + 1])
            sub = W.subset(ss, np.arange(b, e))
            p, l = oracle.sort(sub)
            run_perm[b:e] = p + b
            run_lcp[b:e] = l
        chars, offsets, lengths = to_device(ss)
        rp = torch.from_numpy(run_perm.view(np.int32)).cuda()
        rl = torch.from_numpy(run_lcp.view(np.int32)).cuda()
        perm = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
        lcp = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
        want_perm, want_lcp = oracle.sort(ss)
        for method in (P.MERGE_PAIRWISE, P.MERGE_LOSER_TREE):
            perm.fill_(-1)
            lcp.fill_(-1)
            P.ss_merge_ex(chars, offsets, lengths, ss.fixed_len, rp, rl, rb, perm, lcp, method=method)
            assert np.array_equal(perm.cpu().numpy().view(np.uint32), want_perm), method
            assert np.array_equal(lcp.cpu().numpy().view(np.uint32), want_lcp), method


@pytest.mark.parametrize("K", [2, 4])
def test_batch_runs_then_merge_with_bases(K):
    """The benchmark step: K index-contiguous runs sorted by one ss_sort_batch
    (request-local indices), then ss_merge with each run's index base."""
    import torch
    import paper_1403_2056_gb300 as P
    for ss in (W.url_like(200_000, seed=13), W.dna_windows(150_000, 400_000, 100, seed=14)):
        chars, offsets, lengths = to_device(ss)
        rb = np.array([ss.n * k // K for k in range(K + 1)], np.uint32)
        rperm = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
        rlcp = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
        reqs = []
        for k in range(K):
            b, e = int(rb[k]), int(rb[k + 1])
            reqs.append(dict(chars=chars, offsets=offsets[b:e], lengths=None if lengths is None else lengths[b:e],
                             fixed_len=ss.fixed_len, n=e - b, perm_out=rperm[b:e], lcp_out=rlcp[b:e]))
        P.ss_sort_batch(reqs)
        perm = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
        lcp = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
        P.ss_merge(chars, offsets, lengths, ss.fixed_len, rperm, rlcp, rb, perm, lcp, run_base=rb[:-1])
        want_perm, want_lcp = oracle.sort(ss)
        assert np.array_equal(perm.cpu().numpy().view(np.uint32), want_perm)
        assert np.array_equal(lcp.cpu().numpy().view(np.uint32), want_lcp)


# ------------------------------------------- requests sharing a prefix
def _prefixed(n, prefix, seed, terminated=True, dup_every=0):
    rng = np.random.default_rng(seed)
    tails = [bytes(rng.integers(97, 100, int(rng.integers(0, 14))).astype(np.uint8)) for _ in range(n)]
    strs = [prefix + t for t in tails]
    if dup_every:
        for k in range(dup_every, n, dup_every):
            strs[k] = strs[k - dup_every]
    return W.from_bytes_list(strs, name=f"prefix{len(prefix)}", terminated=terminated)


@pytest.mark.parametrize("plen", [1, 5, 7, 8, 9, 12, 20])
def test_shared_prefix_large_request(plen):
    """Every string of a request above the base-case limit starts with the same
    plen characters (tails over 3 letters, some empty, some duplicates): the
    request starts its first level that deep."""
    _check(_prefixed(30_000, b"q" * (plen - 1) + b"/", seed=plen, dup_every=97))


def test_shared_prefix_explicit_lengths():
    """The same with explicit lengths (bytes 0x01..0xFF, no terminators)."""
    _check(_prefixed(25_000, b"ab\xffcd\x01", seed=3, terminated=False, dup_every=31))


def test_shared_prefix_fixed_length():
    """Fixed-length windows of a text that repeats a 6-character motif with
    rare changes: long shared prefixes inside one request."""
    rng = np.random.default_rng(9)
    text = np.frombuffer(b"ACGTAC" * 200_000, dtype=np.uint8).copy()
    flip = rng.integers(0, text.size, 3000)
    text[flip] = rng.choice(np.frombuffer(b"ACGT", dtype=np.uint8), flip.size)
    offs = (rng.integers(0, (text.size - 40) // 6, 20_000) * 6).astype(np.uint64)
    ss = W.StringSet(chars=text, offsets=offs, lengths=None, fixed_len=40, name="motif40", meta={})
    _check(ss)


def test_batch_with_different_shared_prefixes():
    """Large and small requests in one batch, each with its own shared prefix:
    each request equals the oracle."""
    import torch
    import paper_1403_2056_gb300 as P
    sets = [_prefixed(9_000, b"http://", seed=1), _prefixed(3_000, b"x", seed=2), _prefixed(12_000, b"", seed=3),
            _prefixed(6_000, b"0123456789", seed=4, dup_every=5), W.random_lower(20_000, seed=5)]
    reqs, outs = [], []
    for ss in sets:
        chars, offsets, lengths = to_device(ss)
        perm = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
        lcp = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
        reqs.append(dict(chars=chars, offsets=offsets, lengths=lengths, fixed_len=ss.fixed_len, n=ss.n,
                         perm_out=perm, lcp_out=lcp))
        outs.append((perm, lcp))
    P.ss_sort_batch(reqs)
    torch.cuda.synchronize()
    for ss, (perm, lcp) in zip(sets, outs):
        want_perm, want_lcp = oracle.sort(ss)
        assert np.array_equal(perm.cpu().numpy().view(np.uint32), want_perm), ss.name
        assert np.array_equal(lcp.cpu().numpy().view(np.uint32), want_lcp), ss.name


# ------------------------------------------------------------- tuning
@pytest.mark.parametrize("tuning", [(256, 1), (2048, 9), (32, 3), (65536, 5), (0, 0), (0, 0, 1), (0, 0, 2),
                                    (32, 1, 2), (2048, 9, 1), (0, 0, 0, 0, 2), (0, 0, 0, 0, 6), (0, 0, 0, 0, 0, 64),
                                    (256, 1, 0, 0, 3, 512), (0, 0, 2, 0, 7, 1024)])
def test_tunings_do_not_change_results(tuning):
    """Any tuning gives the same order and LCPs (the oracle's)."""
    import torch
    import paper_1403_2056_gb300 as P
    sets = [W.url_like(60_000, seed=41), W.dna_windows(60_000, 1_200_100, 100, seed=42), W.random_lower(60_000, seed=43),
            W.sinha_dna_like(60_000, seed=44)]
    reqs, outs = [], []
    for ss in sets:
        chars, offsets, lengths = to_device(ss)
        perm = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
        lcp = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
        reqs.append(dict(chars=chars, offsets=offsets, lengths=lengths, fixed_len=ss.fixed_len, n=ss.n,
                         perm_out=perm, lcp_out=lcp))
        outs.append((perm, lcp))
    P.ss_sort_batch_tuned(reqs, [tuning] * len(reqs))
    torch.cuda.synchronize()
    for ss, (perm, lcp) in zip(sets, outs):
        want_perm, want_lcp = oracle.sort(ss)
        assert np.array_equal(perm.cpu().numpy().view(np.uint32), want_perm), (ss.name, tuning)
        assert np.array_equal(lcp.cpu().numpy().view(np.uint32), want_lcp), (ss.name, tuning)


def test_autotune_picks_a_candidate_and_leaves_outputs():
    import torch
    import paper_1403_2056_gb300 as P
    ss = W.url_like(300_000, seed=44)
    chars, offsets, _ = to_device(ss)
    perm = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
    lcp = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
    (ct, ms_step, cls, alpha, md, sm), ms = P.ss_autotune(dict(chars=chars, offsets=offsets, lengths=None,
                                                          fixed_len=0, n=ss.n, perm_out=perm, lcp_out=lcp),
                                                     sample_n=200_000)
    assert ct in (256, 512, 1024, 2048) and ms_step in (1, 3, 5, 9) and cls in (0, 1, 2) and ms > 0
    assert alpha == 0 and md in (0, 6, 7) and sm in (0, 512, 1024)   # NUL-terminated: no alphabet candidate
    torch.cuda.synchronize()
    assert int((perm != -1).sum().item()) == 0 and int((lcp != -1).sum().item()) == 0


def test_autotune_tries_the_alphabet_of_fixed_length_strings():
    """Fixed-length strings over four bytes: the alphabet candidate is found
    from the sample's bytes; whatever is picked sorts like the oracle."""
    import torch
    import paper_1403_2056_gb300 as P
    ss = W.dna_windows(200_000, 4_000_100, 100, seed=45)
    chars, offsets, _ = to_device(ss)
    perm = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
    lcp = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
    q = dict(chars=chars, offsets=offsets, lengths=None, fixed_len=ss.fixed_len, n=ss.n, perm_out=perm, lcp_out=lcp)
    best, ms = P.ss_autotune(q, sample_n=100_000)
    assert best[3] in (0, P.alphabet(b"ACGT")) and ms > 0
    P.ss_sort_batch_tuned([q], [best])
    torch.cuda.synchronize()
    want_perm, want_lcp = oracle.sort(ss)
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), want_perm)
    assert np.array_equal(lcp.cpu().numpy().view(np.uint32), want_lcp)


def test_readme_example():
    """The usage example of the README."""
    import torch
    import paper_1403_2056_gb300 as P
    strs = [b"banana", b"apple", b"cherry", b"apple"]
    chars = torch.tensor(list(b"".join(s + b"\0" for s in strs)), dtype=torch.uint8, device="cuda")
    offsets = torch.tensor(np.cumsum([0] + [len(s) + 1 for s in strs[:-1]]), dtype=torch.int64, device="cuda")
    perm = torch.empty(4, dtype=torch.int32, device="cuda")
    lcp = torch.empty(4, dtype=torch.int32, device="cuda")
    P.ss_sort(chars, offsets, 4, perm, lcp)
    assert perm.tolist() == [1, 3, 0, 2] and lcp.tolist() == [0, 5, 0, 0]


@pytest.mark.parametrize("K", [2, 3, 5, 8])
def test_loser_tree_merge_edge_cases(K):
    """The loser-tree merge on runs of equal strings across runs (ties by run
    order), runs of one string, empty runs between full ones, and runs longer
    than the sparse splitter spacing, against the oracle."""
    import torch
    import paper_1403_2056_gb300 as P
    rng = np.random.default_rng(100 + K)
    words = [b"", b"a", b"ab", b"abc", b"b", b"ba", b"http://x/y", b"http://x/y/z"]
    strs = [words[int(i)] for i in rng.integers(0, len(words), 30_000)]
    ss = W.from_bytes_list(strs)
    sizes = rng.integers(0, 2 * ss.n // K, K)
    sizes[0] = 1
    if K > 2:
        sizes[1] = 0
    cuts = np.minimum(np.cumsum(sizes), ss.n)
    cuts[-1] = ss.n
    rb = np.concatenate([[0], cuts]).astype(np.uint32)
    run_perm = np.empty(ss.n, np.uint32)
    run_lcp = np.empty(ss.n, np.uint32)
    for k in range(K):
        b, e = int(rb[k]), int(rb[k + 1])
        p, l = oracle.sort(W.subset(ss, np.arange(b, e)))
        run_perm[b:e] = p
        run_lcp[b:e] = l
    chars, offsets, lengths = to_device(ss)
    rp = torch.from_numpy(run_perm.view(np.int32)).cuda()
    rl = torch.from_numpy(run_lcp.view(np.int32)).cuda()
    perm = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
    lcp = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
    P.ss_merge_ex(chars, offsets, None, 0, rp, rl, rb, perm, lcp, run_base=rb[:-1], method=P.MERGE_LOSER_TREE)
    want_perm, want_lcp = oracle.sort(ss)
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), want_perm)
    assert np.array_equal(lcp.cpu().numpy().view(np.uint32), want_lcp)


def _sort_tuned(reqs_ss, tunings, asynchronous=False):
    import torch
    import paper_1403_2056_gb300 as P
    reqs, outs = [], []
    for ss in reqs_ss:
        chars, offsets, lengths = to_device(ss)
        perm = torch.full((max(ss.n, 1),), -1, dtype=torch.int32, device="cuda:0")
        lcp = torch.full((max(ss.n, 1),), -1, dtype=torch.int32, device="cuda:0")
        reqs.append(dict(chars=chars, offsets=offsets, lengths=lengths, fixed_len=ss.fixed_len, n=ss.n,
                         perm_out=perm, lcp_out=lcp))
        outs.append((perm, lcp))
    (P.ss_sort_batch_async if asynchronous else P.ss_sort_batch_tuned)(reqs, tunings)
    torch.cuda.synchronize()
    return [(p[:ss.n].cpu().numpy().view(np.uint32), l[:ss.n].cpu().numpy().view(np.uint32))
            for (p, l), ss in zip(outs, reqs_ss)]


@pytest.mark.parametrize("window", [1, 7, 31, 32, 33, 64, 65, 100])
def test_alphabet_compressed_dna_windows(window):
    """Alphabet compression (2-bit codes, 32 characters per key) on DNA windows
    whose length falls below, on and across key boundaries, with many
    duplicate windows (short text), against the oracle."""
    import paper_1403_2056_gb300 as P
    ss = W.dna_windows(60_000, 3_000 + window, window, seed=window)
    (perm, lcp), = _sort_tuned([ss], [(0, 0, 0, P.alphabet(b"ACGT"))])
    want_perm, want_lcp = oracle.sort(ss)
    assert np.array_equal(perm, want_perm)
    assert np.array_equal(lcp, want_lcp)


def test_alphabet_compressed_small_alphabets_and_mixed_batch():
    """One batch mixing compressed requests (alphabets of 2 and 4 bytes, windows
    over one text) with plain ones (the same windows without compression, a
    URL-like set, tiny requests): every request equals the oracle's sort."""
    import paper_1403_2056_gb300 as P
    rng = np.random.default_rng(7)
    text = np.frombuffer(b"AC", np.uint8)[rng.integers(0, 2, 20_000)]
    two = W.StringSet(np.concatenate([text, np.zeros(16, np.uint8)]),
                      rng.integers(0, text.size - 40, 30_000).astype(np.uint64), None, 40, "ac_windows")
    dna = W.dna_windows(50_000, 200_000, 100, seed=11)
    url = W.url_like(40_000, seed=12)
    tiny = W.dna_windows(3, 50, 20, seed=13)
    sets = [two, dna, url, dna, tiny]
    tun = [(0, 0, 0, P.alphabet(b"AC")), (0, 0, 0, P.alphabet(b"ACGT")), (0, 0, 0, 0), (0, 0, 0, 0),
           (0, 0, 0, P.alphabet(b"ACGT"))]
    for (perm, lcp), ss in zip(_sort_tuned(sets, tun), sets):
        want_perm, want_lcp = oracle.sort(ss)
        assert np.array_equal(perm, want_perm), ss.name
        assert np.array_equal(lcp, want_lcp), ss.name


def test_async_sort_returns_before_the_sort_completes():
    """ss_sort_batch_async only queues work: the recursion is driven by the
    device, so the call returns well before the sort is done on the stream,
    and the outputs are complete (and equal the oracle's) once the stream
    reaches an event recorded after the call."""
    import time
    import torch
    import paper_1403_2056_gb300 as P
    ss = W.url_like(3_000_000, seed=73)
    chars, offsets, _ = to_device(ss)
    perm = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
    lcp = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
    stream = torch.cuda.current_stream()
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda:0")
    req = [dict(chars=chars, offsets=offsets, n=ss.n, perm_out=perm, lcp_out=lcp, status_out=status)]
    P.ss_sort_batch_async(req, stream=stream)   # warm-up: pool growth, attributes
    torch.cuda.synchronize()
    calls, gpu = [], []
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t0 = time.perf_counter()
        P.ss_sort_batch_async(req, stream=stream)
        calls.append((time.perf_counter() - t0) * 1e3)
        e1.record(stream)
        e1.synchronize()
        gpu.append(e0.elapsed_time(e1))
    assert min(calls) < 0.5 * min(gpu), (calls, gpu)
    assert int(status.item()) == 0
    want_perm, want_lcp = oracle.sort(ss)
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), want_perm)
    assert np.array_equal(lcp.cpu().numpy().view(np.uint32), want_lcp)


def test_device_and_host_driven_levels_agree():
    """Levels driven by the device scheduler (ss_sort_batch_async) and by the
    host (ss_sort_batch_tuned) give the same arrays, on a request that needs
    many levels (long shared prefixes), URL-like and DNA-like requests, with
    and without alphabet compression, and a batch of tiny requests."""
    import paper_1403_2056_gb300 as P
    sets = [W.from_bytes_list([b"p" * 200 + str(i % 977).encode() * 3 for i in range(20_000)]),
            W.url_like(200_000, seed=74), W.dna_windows(100_000, 150_000, 100, seed=75),
            W.dna_windows(100_000, 150_000, 100, seed=76)] + [W.random_lower(k, seed=k) for k in (0, 1, 2, 31, 300)]
    tun = [(0, 0, 0, 0)] * 3 + [(0, 0, 0, P.alphabet(b"ACGT"))] + [(0, 0, 0, 0)] * 5
    res = [_sort_tuned(sets, tun), _sort_tuned(sets, tun, asynchronous=True)]
    for (p0, l0), (p1, l1), ss in zip(res[0], res[1], sets):
        assert np.array_equal(p0, p1) and np.array_equal(l0, l1), ss.name
        want_perm, want_lcp = oracle.sort(ss)
        assert np.array_equal(p0, want_perm) and np.array_equal(l0, want_lcp), ss.name


# ------------------------------------------------------- sort caches
def _check_caches(ss, perm, lcp, off, ck, ckd, base=0):
    """off = the string's offset; ck = 8 bytes of the string from ckd
    (big-endian, zero past its end); ckd <= lcp < ckd + 8 or the string ends
    before ckd + 8; position 0 at depth 0 (the sort-cache contract)."""
    assert ckd[0] == 0
    for p in range(len(perm)):
        i = int(perm[p]) + base
        s = ss.string(i)
        d = int(ckd[p])
        assert int(off[p]) == int(ss.offsets[i]), p
        want = int.from_bytes((s[d:d + 8] + bytes(8))[:8], "big")
        assert int(ck[p]) == want, (p, d)
        assert d <= int(lcp[p]), (p, d, int(lcp[p]))
        assert int(lcp[p]) < d + 8 or len(s) < d + 8, (p, d, int(lcp[p]))


@pytest.mark.parametrize("make", [lambda: W.url_like(40_000, seed=61), lambda: W.random_lower(30_000, seed=62),
                                  lambda: W.dna_windows(30_000, 600_100, 100, seed=63),
                                  lambda: W.sinha_dna_like(30_000, seed=64),
                                  lambda: W.from_bytes_list([b"ab"[i % 2:i % 2 + 1] * (i % 7) for i in range(5000)]),
                                  lambda: W.from_bytes_list([bytes([65 + i % 3]) * (i % 40) for i in range(3000)],
                                                            terminated=False)])
def test_sort_caches_and_cached_merge(make):
    """ss_sort_batch_cached writes caches that satisfy their contract (checked
    against the strings, every position), and ss_merge_cached of the runs from
    them equals the oracle's sort of the whole set."""
    import torch
    import paper_1403_2056_gb300 as P
    ss = make()
    n, K = ss.n, 3
    rb = np.array([n * k // K for k in range(K + 1)], np.uint32)
    chars, offsets, lengths = to_device(ss)
    rperm = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
    rlcp = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
    off = torch.full((n,), -1, dtype=torch.int64, device="cuda:0")
    ck = torch.full((n,), -1, dtype=torch.int64, device="cuda:0")
    ckd = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
    reqs, caches = [], []
    for k in range(K):
        b, e = int(rb[k]), int(rb[k + 1])
        reqs.append(dict(chars=chars, offsets=offsets[b:e], lengths=None if lengths is None else lengths[b:e],
                         fixed_len=ss.fixed_len, n=e - b, perm_out=rperm[b:e], lcp_out=rlcp[b:e]))
        caches.append((off[b:e], ck[b:e], ckd[b:e]))
    P.ss_sort_batch_cached(reqs, caches)
    torch.cuda.synchronize()
    hp, hl = rperm.cpu().numpy().view(np.uint32), rlcp.cpu().numpy().view(np.uint32)
    ho, hk, hd = off.cpu().numpy().view(np.uint64), ck.cpu().numpy().view(np.uint64), ckd.cpu().numpy().view(np.uint32)
    for k in range(K):
        b, e = int(rb[k]), int(rb[k + 1])
        want_p, want_l = oracle.sort(W.subset(ss, np.arange(b, e)))
        assert np.array_equal(hp[b:e], want_p) and np.array_equal(hl[b:e], want_l), k
        _check_caches(ss, hp[b:e], hl[b:e], ho[b:e], hk[b:e], hd[b:e], base=b)
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
    lcp = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
    P.ss_merge_cached(chars, offsets, lengths, ss.fixed_len, rperm, rlcp, off, ck, ckd, rb, perm, lcp,
                      run_base=rb[:-1])
    torch.cuda.synchronize()
    want_perm, want_lcp = oracle.sort(ss)
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), want_perm)
    assert np.array_equal(lcp.cpu().numpy().view(np.uint32), want_lcp)


def test_sort_caches_of_tiny_and_single_requests():
    """Requests of 1, 2 and 33 strings (init, warp and CTA paths) write their caches."""
    import torch
    import paper_1403_2056_gb300 as P
    sets = [W.random_lower(1, seed=65), W.random_lower(2, seed=66), W.url_like(33, seed=67), W.url_like(3000, seed=68)]
    reqs, caches, outs = [], [], []
    for ss in sets:
        chars, offsets, lengths = to_device(ss)
        t = [torch.full((ss.n,), -1, dtype=d, device="cuda:0") for d in (torch.int32, torch.int32, torch.int64,
                                                                          torch.int64, torch.int32)]
        reqs.append(dict(chars=chars, offsets=offsets, lengths=lengths, fixed_len=ss.fixed_len, n=ss.n,
                         perm_out=t[0], lcp_out=t[1]))
        caches.append((t[2], t[3], t[4]))
        outs.append(t)
    P.ss_sort_batch_cached(reqs, caches)
    torch.cuda.synchronize()
    for ss, t in zip(sets, outs):
        p, l = t[0].cpu().numpy().view(np.uint32), t[1].cpu().numpy().view(np.uint32)
        want_p, want_l = oracle.sort(ss)
        assert np.array_equal(p, want_p) and np.array_equal(l, want_l)
        _check_caches(ss, p, l, t[2].cpu().numpy().view(np.uint64), t[3].cpu().numpy().view(np.uint64),
                      t[4].cpu().numpy().view(np.uint32))
