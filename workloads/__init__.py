"""Seeded synthetic string sets shaped like the paper's inputs (Section 7.2, Table 3).

This module only draws random bytes and lays them out; it holds none of the
sorting arithmetic.  Both the CPU oracle tests and the CUDA path read the
arrays it returns, so one seed gives both sides the same input.

Every generator returns a :class:`StringSet`:

* ``chars``   -- uint8 array holding all string bytes,
* ``offsets`` -- uint64[n], the first byte of string i inside ``chars``,
* ``lengths`` -- uint32[n] or None; when None the strings are either
  NUL-terminated (``fixed_len == 0``) or all exactly ``fixed_len`` bytes long
  and not terminated (DNA windows of one shared text).

Random numbers come from ``numpy.random.default_rng(seed)`` (PCG64), which
gives the same stream on x86-64 and aarch64.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

__all__ = [
    "StringSet",
    "from_bytes_list",
    "random_lower",
    "url_like",
    "dna_windows",
    "no_lcp",
    "sinha_dna_like",
    "paper_random",
    "subset",
]


@dataclass
class StringSet:
    chars: np.ndarray
    offsets: np.ndarray
    lengths: Optional[np.ndarray] = None
    fixed_len: int = 0
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0])

    @property
    def terminated(self) -> bool:
        return self.lengths is None and self.fixed_len == 0

    def string(self, i: int) -> bytes:
        """Bytes of string i without its terminator (host-side helper)."""
        off = int(self.offsets[i])
        if self.lengths is not None:
            return self.chars[off: off + int(self.lengths[i])].tobytes()
        if self.fixed_len:
            return self.chars[off: off + self.fixed_len].tobytes()
        end = off
        buf = self.chars
        while buf[end] != 0:
            end += 1
        return buf[off:end].tobytes()

    def strings(self) -> list:
        return [self.string(i) for i in range(self.n)]

    def all_lengths(self) -> np.ndarray:
        """uint64 length of every string (terminator excluded)."""
        if self.lengths is not None:
            return self.lengths.astype(np.uint64)
        if self.fixed_len:
            return np.full(self.n, self.fixed_len, dtype=np.uint64)
        zeros = np.flatnonzero(self.chars == 0).astype(np.uint64)
        # first terminator at or after each offset
        pos = np.searchsorted(zeros, self.offsets)
        return zeros[pos] - self.offsets

    @property
    def total_bytes(self) -> int:
        return int(self.chars.nbytes)


def _pad(chars: np.ndarray) -> np.ndarray:
    """Pad the byte buffer to a multiple of 8 with zeros (aligned words stay in bounds)."""
    extra = (-chars.shape[0]) % 8
    if extra:
        chars = np.concatenate([chars, np.zeros(extra, dtype=np.uint8)])
    return chars


def from_bytes_list(strs, name: str = "list", terminated: bool = True) -> StringSet:
    """Lay out a Python list of byte strings contiguously.

    terminated=True: each string is followed by a 0 byte (strings must not
    contain 0).  terminated=False: lengths are given explicitly and strings may
    hold any byte, including 0.
    """
    strs = [bytes(s) for s in strs]
    n = len(strs)
    if terminated:
        for s in strs:
            if 0 in s:
                raise ValueError("NUL byte inside a terminated string")
        lens = np.array([len(s) + 1 for s in strs], dtype=np.uint64)
    else:
        lens = np.array([len(s) for s in strs], dtype=np.uint64)
    offsets = np.zeros(n, dtype=np.uint64)
    if n:
        offsets[1:] = np.cumsum(lens)[:-1]
    blob = b"".join((s + b"\0") if terminated else s for s in strs)
    chars = _pad(np.frombuffer(blob, dtype=np.uint8).copy() if blob else np.zeros(0, np.uint8))
    if chars.shape[0] == 0:
        chars = np.zeros(8, dtype=np.uint8)
    if terminated:
        return StringSet(chars, offsets, None, 0, name)
    return StringSet(chars, offsets, np.array([len(s) for s in strs], dtype=np.uint32), 0, name)


def _layout_terminated(lengths: np.ndarray):
    """offsets for contiguous NUL-terminated strings of the given lengths."""
    n = lengths.shape[0]
    stride = lengths.astype(np.uint64) + 1
    offsets = np.zeros(n, dtype=np.uint64)
    if n:
        np.cumsum(stride[:-1], out=offsets[1:])
    total = int(stride.sum()) if n else 0
    return offsets, total


def _fill_uniform_bytes(rng, chars, offsets, lengths, alphabet: np.ndarray, chunk=1 << 22):
    """Fill bytes [off, off+len) of every string with i.i.d. letters of ``alphabet``."""
    n = offsets.shape[0]
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        lens = lengths[s:e].astype(np.int64)
        tot = int(lens.sum())
        if tot == 0:
            continue
        sid = np.repeat(np.arange(e - s), lens)
        starts = np.zeros(e - s, dtype=np.int64)
        np.cumsum(lens[:-1], out=starts[1:])
        pos_in = np.arange(tot, dtype=np.int64) - starts[sid]
        dst = offsets[s:e].astype(np.int64)[sid] + pos_in
        chars[dst] = alphabet[rng.integers(0, alphabet.shape[0], tot)]


def random_lower(n: int = 200_000, seed: int = 1, min_len: int = 8, max_len: int = 32) -> StringSet:
    """Plain single sort: length U[min_len, max_len], bytes U['a'..'z'], NUL-terminated."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(min_len, max_len + 1, n).astype(np.uint64)
    offsets, total = _layout_terminated(lengths)
    chars = np.zeros(total, dtype=np.uint8)
    alpha = np.arange(ord("a"), ord("z") + 1, dtype=np.uint8)
    _fill_uniform_bytes(rng, chars, offsets, lengths, alpha)
    return StringSet(_pad(chars), offsets, None, 0, f"random_lower(n={n},seed={seed})")


def paper_random(n: int, seed: int = 11) -> StringSet:
    """The paper's Random set (Section 7.2): length U[0,20), bytes U[33,127), NUL-terminated."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(0, 20, n).astype(np.uint64)
    offsets, total = _layout_terminated(lengths)
    chars = np.zeros(total, dtype=np.uint8)
    alpha = np.arange(33, 127, dtype=np.uint8)
    _fill_uniform_bytes(rng, chars, offsets, lengths, alpha)
    return StringSet(_pad(chars), offsets, None, 0, f"paper_random(n={n},seed={seed})")


def sinha_dna_like(n: int, seed: int = 12, length: int = 9) -> StringSet:
    """Strings of ``length`` letters over {A,C,G,T}, NUL-terminated (shape of Sinha's DNA set)."""
    rng = np.random.default_rng(seed)
    lengths = np.full(n, length, dtype=np.uint64)
    offsets, total = _layout_terminated(lengths)
    chars = np.zeros(total, dtype=np.uint8)
    alpha = np.frombuffer(b"ACGT", dtype=np.uint8)
    _fill_uniform_bytes(rng, chars, offsets, lengths, alpha)
    return StringSet(_pad(chars), offsets, None, 0, f"sinha_dna_like(n={n},seed={seed})")


_URL_HOST_ALPHA = np.frombuffer(b"abcdefghijklmnopqrstuvwxyz.", dtype=np.uint8)
_URL_PATH_ALPHA = np.frombuffer(b"abcdefghijklmnopqrstuvwxyz0123456789/", dtype=np.uint8)
_HTTP = np.frombuffer(b"http://", dtype=np.uint8)


def url_like(n: int = 10_000_000, seed: int = 2, hosts: int = 2000, zipf_s: float = 1.1,
             dup_frac: float = 0.05, chunk: int = 1 << 20) -> StringSet:
    """URL-like shared-prefix set.

    'http://' + host + 1..6 path segments ('/' + 3..12 chars over [a-z0-9/]).
    The host pool (``hosts`` names, length U[8,20] over [a-z.]) is drawn once;
    string i picks host rank k with probability proportional to k^-zipf_s.
    With probability ``dup_frac`` string i is instead an exact copy of a
    uniformly chosen earlier string.  NUL-terminated, contiguous.
    """
    rng = np.random.default_rng(seed)
    # host pool
    hlen = rng.integers(8, 21, hosts).astype(np.int64)
    hstart = np.zeros(hosts, dtype=np.int64)
    np.cumsum(hlen[:-1], out=hstart[1:])
    hbytes = _URL_HOST_ALPHA[rng.integers(0, _URL_HOST_ALPHA.shape[0], int(hlen.sum()))]
    p = np.arange(1, hosts + 1, dtype=np.float64) ** (-zipf_s)
    p /= p.sum()
    host = rng.choice(hosts, size=n, p=p).astype(np.int64)
    nseg = rng.integers(1, 7, n).astype(np.int64)
    seglen = rng.integers(3, 13, (n, 6)).astype(np.int64)
    seglen[np.arange(6)[None, :] >= nseg[:, None]] = 0
    seg_tot = (seglen + (seglen > 0)).sum(axis=1)
    # duplicates: copy of a uniformly chosen earlier string, chains resolved
    origin = np.arange(n, dtype=np.int64)
    dup = rng.random(n) < dup_frac
    if n:
        dup[0] = False
    di = np.flatnonzero(dup)
    origin[di] = (rng.random(di.shape[0]) * di).astype(np.int64)
    for _ in range(64):
        nxt = origin[origin]
        if np.array_equal(nxt, origin):
            break
        origin = nxt
    lengths = (7 + hlen[host] + seg_tot)[origin].astype(np.uint64)
    offsets, total = _layout_terminated(lengths)
    chars = np.zeros(total, dtype=np.uint8)
    off64 = offsets.astype(np.int64)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        idx = np.arange(s, e)
        fresh = idx[origin[s:e] == idx]
        # fresh strings: generate bytes
        L = lengths[fresh].astype(np.int64)
        tot = int(L.sum())
        sid = np.repeat(np.arange(fresh.shape[0]), L)
        st = np.zeros(fresh.shape[0], dtype=np.int64)
        if fresh.shape[0]:
            np.cumsum(L[:-1], out=st[1:])
        pos = np.arange(tot, dtype=np.int64) - st[sid]
        gi = fresh[sid]
        out = _URL_PATH_ALPHA[rng.integers(0, _URL_PATH_ALPHA.shape[0], tot)]
        m = pos < 7
        out[m] = _HTTP[pos[m]]
        hl = hlen[host[gi]]
        m = (pos >= 7) & (pos < 7 + hl)
        out[m] = hbytes[hstart[host[gi[m]]] + pos[m] - 7]
        chars[off64[gi] + pos] = out
        # slashes at segment starts
        base = off64[fresh] + 7 + hlen[host[fresh]]
        run = np.zeros(fresh.shape[0], dtype=np.int64)
        for k in range(6):
            sl = seglen[fresh, k]
            has = sl > 0
            chars[(base + run)[has]] = ord("/")
            run += np.where(has, sl + 1, 0)
        # copies: origin is earlier, already written
        cp = idx[origin[s:e] != idx]
        if cp.shape[0]:
            L = lengths[cp].astype(np.int64)
            tot = int(L.sum())
            sid = np.repeat(np.arange(cp.shape[0]), L)
            st = np.zeros(cp.shape[0], dtype=np.int64)
            np.cumsum(L[:-1], out=st[1:])
            pos = np.arange(tot, dtype=np.int64) - st[sid]
            chars[off64[cp[sid]] + pos] = chars[off64[origin[cp[sid]]] + pos]
    ss = StringSet(_pad(chars), offsets, None, 0, f"url_like(n={n},seed={seed})")
    ss.meta["mean_len"] = float(lengths.mean()) if n else 0.0
    ss.meta["dup_frac"] = float(dup.mean()) if n else 0.0
    return ss


def dna_windows(n: int = 20_000_000, text_len: int = 400_000_000, window: int = 100,
                seed: int = 3) -> StringSet:
    """DNA-like windows: a text of ``text_len`` bytes U{A,C,G,T} and ``n`` windows of
    ``window`` bytes starting at uniform offsets in [0, text_len - window].
    The windows are not terminated: every string is exactly ``window`` bytes."""
    rng = np.random.default_rng(seed)
    alpha = np.frombuffer(b"ACGT", dtype=np.uint8)
    chars = np.empty(text_len, dtype=np.uint8)
    step = 1 << 26
    for s in range(0, text_len, step):
        e = min(text_len, s + step)
        chars[s:e] = alpha[rng.integers(0, 4, e - s, dtype=np.uint8)]
    offsets = rng.integers(0, text_len - window + 1, n).astype(np.uint64)
    return StringSet(_pad(chars), offsets, None, window, f"dna_windows(n={n},T={text_len},seed={seed})")


def no_lcp(n: int = 64 * 1024 * 1024, length: int = 16, seed: int = 5, chunk: int = 1 << 23) -> StringSet:
    """Near-zero-LCP job: n strings of ``length`` bytes U[1,255], NUL-terminated, stride length+1."""
    rng = np.random.default_rng(seed)
    stride = length + 1
    chars = np.zeros(n * stride, dtype=np.uint8)
    view = chars.reshape(n, stride) if n else chars.reshape(0, stride)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        view[s:e, :length] = rng.integers(1, 256, (e - s, length), dtype=np.uint8)
    offsets = (np.arange(n, dtype=np.uint64) * np.uint64(stride))
    return StringSet(_pad(chars), offsets, None, 0, f"no_lcp(n={n},len={length},seed={seed})")


def subset(ss: StringSet, idx: np.ndarray) -> StringSet:
    """Strings ``idx`` of ``ss`` re-indexed 0..len(idx)-1, sharing the same byte buffer."""
    idx = np.asarray(idx, dtype=np.int64)
    lengths = None if ss.lengths is None else ss.lengths[idx].copy()
    return StringSet(ss.chars, ss.offsets[idx].copy(), lengths, ss.fixed_len, ss.name + "[subset]")
