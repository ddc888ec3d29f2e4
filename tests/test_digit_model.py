"""Host model of the base case's counting first round (ss_base.cuh): the two
digits it distributes by must lie in [0, 2^B) and be monotone in the key, or
the counting pass would not sort.  The model repeats the kernel's arithmetic
step for step (float32 with round-to-nearest, as the kernel's float division
and conversions are): the interpolation digit over the segment's key range in
fixed point, and the rank digit of keys of a small alphabet.  It also checks
the reason for the interpolation digit: on keys spread over a bucket between
two splitters, the bits after the common prefix overfill a digit far more
often than the interpolation digit does.  Not the oracle; shares no code
with it."""
import numpy as np
import pytest

M64 = (1 << 64) - 1


def _bits(m):
    b = 1
    while (1 << b) < m:
        b += 1
    return b


def interp_digit_fn(kmin, kmax, B):
    """the kernel's fixed-point interpolation digit for keys in [kmin, kmax]"""
    span = kmax - kmin
    L = 64 - span.bit_length()                      # clz(span), span > 0
    sh = ((span << L) & M64) >> 32
    q = np.float32(np.float32(np.float32(2.0 ** 44) / (np.float32(sh) + np.float32(1.0)))
                   * np.float32(np.float32(1.0) - np.float32(1.0) / np.float32(1048576.0)))
    M = int(q)                                      # round toward zero
    return lambda k: (((((k - kmin) << L) & M64) >> 32) * M) >> (44 - B)


def rank_digit_fn(keys, B):
    """the kernel's rank digit: bytes from the first differing one, each
    replaced by its rank among the byte values the keys use there"""
    x = 0
    for k in keys:
        x |= k ^ keys[0]
    c0 = (64 - x.bit_length()) >> 3
    used = sorted({(k >> (56 - 8 * j)) & 0xFF for k in keys for j in range(c0, 8)})
    rank = {v: i for i, v in enumerate(used)}
    bw = _bits(len(used))

    def d(k):
        dd, nbits, j = 0, 0, c0
        while j < 8 and nbits < B:
            dd = (dd << bw) | rank[(k >> (56 - 8 * j)) & 0xFF]
            nbits += bw
            j += 1
        return dd >> (nbits - B) if nbits >= B else dd << (B - nbits)
    return d


@pytest.mark.parametrize("seed", range(6))
def test_interpolation_digit_in_range_and_monotone(seed):
    rng = np.random.default_rng(seed)
    spans = [1, 2, 3, 255, (1 << 24) - 1, 1 << 24, (1 << 32) + 1, 1 << 63, M64] + \
            [int(s) for s in rng.integers(1, 1 << 63, 40, dtype=np.uint64)]
    for span in spans:
        kmin = int(rng.integers(0, (M64 - span) >> 1 if span < M64 else 1, dtype=np.uint64)) if span < M64 else 0
        kmax = kmin + span
        for m in (2, 33, 300, 1024, 2048):
            B = _bits(m)
            d = interp_digit_fn(kmin, kmax, B)
            ks = sorted({kmin, kmax, kmin + span // 2} | {kmin + int(r) % (span + 1)
                                                           for r in rng.integers(0, 1 << 63, 64, dtype=np.uint64)})
            ds = [d(k) for k in ks]
            assert all(0 <= v < (1 << B) for v in ds), (span, B)
            assert all(a <= b for a, b in zip(ds, ds[1:])), (span, B)
            # the whole digit range is used: the largest key lands in the top digit but one at most
            assert d(kmax) >= (1 << B) - 2 or span < (1 << B), (span, B, d(kmax))


def test_rank_digit_in_range_and_monotone():
    rng = np.random.default_rng(7)
    for trial in range(30):
        alphabet = rng.choice(np.arange(1, 256), size=int(rng.integers(2, 17)), replace=False)
        m = int(rng.integers(2, 2049))
        prefix = int(rng.integers(0, 4))
        keys = []
        for _ in range(m):
            bs = [65] * prefix + [int(v) for v in rng.choice(alphabet, size=8 - prefix)]
            keys.append(int.from_bytes(bytes(bs), "big"))
        if len(set(keys)) == 1:
            continue
        B = _bits(m)
        d = rank_digit_fn(keys, B)
        ks = sorted(set(keys))
        ds = [d(k) for k in ks]
        assert all(0 <= v < (1 << B) for v in ds)
        assert all(a <= b for a, b in zip(ds, ds[1:]))


def test_interpolation_digit_fills_buckets_the_prefix_bits_overfill():
    """Keys uniform in a bucket between two random splitters: the digit of
    the bits after the keys' common prefix overfills (> 8 strings) in a
    large share of segments, the interpolation digit almost never."""
    rng = np.random.default_rng(11)
    fail_bits = fail_interp = 0
    T = 120
    for _ in range(T):
        m = int(rng.integers(257, 2049))
        width = int(rng.integers(1 << 40, 1 << 44))
        lo = int(rng.integers(0, 1 << 62))
        keys = [lo + int(r) % width for r in rng.integers(0, 1 << 63, m, dtype=np.uint64)]
        B = _bits(m)
        x = 0
        for k in keys:
            x |= k ^ keys[0]
        cp = 64 - x.bit_length()
        cnt = np.bincount([((k << cp) & M64) >> (64 - B) for k in keys], minlength=1 << B)
        fail_bits += int(cnt.max() > 8)
        d = interp_digit_fn(min(keys), max(keys), B)
        cnt = np.bincount([d(k) for k in keys], minlength=1 << B)
        fail_interp += int(cnt.max() > 8)
    assert fail_bits > T // 5, fail_bits
    assert fail_interp <= 1, fail_interp
