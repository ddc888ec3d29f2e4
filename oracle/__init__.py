"""CPU correctness oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use this package.  The CUDA library never imports or links it, and it
imports nothing from the CUDA library.

The arithmetic lives in ``oracle.c`` (plain C, compiled with gcc on first use
into ``oracle/_build/liboracle.so``); this module only marshals numpy arrays.
See ``oracle.c`` for the passage of the paper each function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u8p = C.POINTER(C.c_uint8)
_u16p = C.POINTER(C.c_uint16)
_u32p = C.POINTER(C.c_uint32)
_u64p = C.POINTER(C.c_uint64)


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (portable flags: same results on x86-64 and aarch64)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


_PAR_SRC = os.path.join(_HERE, "parallel.cpp")
_PAR_SO = os.path.join(_OUT_DIR, "libparallel.so")
_par = None


def build_parallel(force: bool = False) -> str:
    """Compile parallel.cpp (the parallel library-sort baseline) with g++ and OpenMP."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_PAR_SO) or os.path.getmtime(_PAR_SO) < os.path.getmtime(_PAR_SRC):
        tmp = _PAR_SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-Wall", "-shared", "-fPIC", "-o", tmp,
                               _PAR_SRC])
        os.replace(tmp, _PAR_SO)
    return _PAR_SO


def sort_parallel(ss, threads: int = 0):
    """(perm, lcp, threads used): the oracle's order by a parallel library
    stable sort on `threads` host threads (0: all), naive LCPs; a CPU
    baseline for comparison, checked against sort() by the tests."""
    global _par
    with _lock:
        if _par is None:
            lib = C.CDLL(build_parallel())
            lib.orc_sort_parallel.argtypes = [_u8p, _u64p, _u32p, C.c_uint32, C.c_uint64, _u32p, _u32p, C.c_int]
            lib.orc_sort_parallel.restype = C.c_int
            _par = lib
    keep, a = _set(ss)
    perm = np.empty(ss.n, np.uint32)
    lcp = np.empty(ss.n, np.uint32)
    used = _par.orc_sort_parallel(*a, ss.n, _p(perm, _u32p), _p(lcp, _u32p), int(threads))
    return perm, lcp, int(used)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            set_args = [_u8p, _u64p, _u32p, C.c_uint32]
            lib.orc_sort.argtypes = set_args + [C.c_uint64, _u32p, _u32p]
            lib.orc_sort.restype = C.c_int
            lib.orc_lcp_of.argtypes = set_args + [C.c_uint64, _u32p, _u32p]
            lib.orc_cmp.argtypes = set_args + [C.c_uint64, C.c_uint64]
            lib.orc_cmp.restype = C.c_int
            lib.orc_stats.argtypes = set_args + [C.c_uint64, _u32p, _u32p, _u64p, _u64p, _u64p]
            lib.orc_chars_h.argtypes = set_args + [C.c_uint64, C.c_uint64]
            lib.orc_chars_h.restype = C.c_uint64
            lib.orc_chars_h_all.argtypes = set_args + [C.c_uint64, _u64p, _u64p]
            lib.orc_s5_tree.argtypes = [_u64p, C.c_uint32, _u64p]
            lib.orc_s5_classify.argtypes = [_u64p, C.c_uint64, _u64p, C.c_uint32, _u16p]
            lib.orc_s5_classify_equal.argtypes = [_u64p, C.c_uint64, _u64p, C.c_uint32, _u16p]
            lib.orc_s5_distribute.argtypes = [_u16p, C.c_uint64, C.c_uint32, _u64p, _u64p]
            lib.orc_s5_pick.argtypes = [_u64p, C.c_uint64, C.c_uint32, _u64p]
            lib.orc_lcp_compare.argtypes = set_args + [C.c_uint64] * 4 + [_u64p]
            lib.orc_lcp_compare.restype = C.c_uint64
            lib.orc_lcp_merge2.argtypes = set_args + [_u32p, _u32p, C.c_uint64, _u32p, _u32p,
                                                      C.c_uint64, _u32p, _u32p]
            lib.orc_lcp_merge2.restype = C.c_uint64
            lib.orc_lcp_mergek.argtypes = set_args + [_u32p, _u32p, _u64p, C.c_uint32, _u32p, _u32p]
            lib.orc_lcp_mergek.restype = C.c_uint64
            lib.orc_lcp_insertion.argtypes = set_args + [_u32p, _u32p, C.c_uint64, C.c_uint64]
            lib.orc_lcp_insertion.restype = C.c_uint64
            lib.orc_check_sorted.argtypes = set_args + [C.c_uint64, _u32p, _u32p, _u64p]
            lib.orc_check_sorted.restype = C.c_uint64
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _set(ss):
    chars = _c(ss.chars, np.uint8)
    offs = _c(ss.offsets, np.uint64)
    lens = None if ss.lengths is None else _c(ss.lengths, np.uint32)
    keep = (chars, offs, lens)
    return keep, [_p(chars, _u8p), _p(offs, _u64p), _p(lens, _u32p), C.c_uint32(int(ss.fixed_len))]


def sort(ss):
    """(perm, lcp): lexicographic order, ties by index; lcp[0] = 0 (Section 2)."""
    lib = _load()
    keep, a = _set(ss)
    n = ss.n
    perm = np.empty(n, np.uint32)
    lcp = np.empty(n, np.uint32)
    lib.orc_sort(*a, n, _p(perm, _u32p), _p(lcp, _u32p))
    return perm, lcp


def lcp_of(ss, perm):
    """Naive LCP array of the order ``perm``."""
    lib = _load()
    keep, a = _set(ss)
    perm = _c(perm, np.uint32)
    lcp = np.empty(perm.shape[0], np.uint32)
    lib.orc_lcp_of(*a, perm.shape[0], _p(perm, _u32p), _p(lcp, _u32p))
    return lcp


def cmp(ss, a_idx: int, b_idx: int) -> int:
    lib = _load()
    keep, a = _set(ss)
    return int(lib.orc_cmp(*a, a_idx, b_idx))


def stats(ss, perm, lcp):
    """(L, D, N) of Section 2 for a sorted order with its LCP array."""
    lib = _load()
    keep, a = _set(ss)
    perm = _c(perm, np.uint32)
    lcp = _c(lcp, np.uint32)
    L, D, N = C.c_uint64(), C.c_uint64(), C.c_uint64()
    lib.orc_stats(*a, perm.shape[0], _p(perm, _u32p), _p(lcp, _u32p), C.byref(L), C.byref(D), C.byref(N))
    return int(L.value), int(D.value), int(N.value)


def chars_h(ss, i: int, h: int) -> int:
    lib = _load()
    keep, a = _set(ss)
    return int(lib.orc_chars_h(*a, i, h))


def chars_h_all(ss, depth):
    lib = _load()
    keep, a = _set(ss)
    depth = _c(depth, np.uint64)
    keys = np.empty(ss.n, np.uint64)
    lib.orc_chars_h_all(*a, ss.n, _p(depth, _u64p), _p(keys, _u64p))
    return keys


def s5_tree(x):
    lib = _load()
    x = _c(x, np.uint64)
    t = np.empty(x.shape[0], np.uint64)
    lib.orc_s5_tree(_p(x, _u64p), x.shape[0], _p(t, _u64p))
    return t


def s5_classify(keys, x):
    lib = _load()
    keys = _c(keys, np.uint64)
    x = _c(x, np.uint64)
    b = np.empty(keys.shape[0], np.uint16)
    lib.orc_s5_classify(_p(keys, _u64p), keys.shape[0], _p(x, _u64p), x.shape[0], _p(b, _u16p))
    return b


def s5_classify_equal(keys, x):
    """S5-Equal: equality test at every node of one descent (Section 4.4)."""
    lib = _load()
    keys = _c(keys, np.uint64)
    x = _c(x, np.uint64)
    b = np.empty(keys.shape[0], np.uint16)
    lib.orc_s5_classify_equal(_p(keys, _u64p), keys.shape[0], _p(x, _u64p), x.shape[0], _p(b, _u16p))
    return b


def s5_distribute(bucket, v: int):
    """(bucket_begin[2v+2], out): counts, prefix sum and stable redistribution."""
    lib = _load()
    bucket = _c(bucket, np.uint16)
    bb = np.empty(2 * v + 2, np.uint64)
    out = np.empty(bucket.shape[0], np.uint64)
    lib.orc_s5_distribute(_p(bucket, _u16p), bucket.shape[0], v, _p(bb, _u64p), _p(out, _u64p))
    return bb, out


def s5_pick(sorted_sample, v: int):
    lib = _load()
    s = _c(sorted_sample, np.uint64)
    x = np.empty(v, np.uint64)
    lib.orc_s5_pick(_p(s, _u64p), s.shape[0], v, _p(x, _u64p))
    return x


def lcp_compare(ss, a_idx, ha, b_idx, hb):
    """((x, h_x, y, h'), comparisons) of LCP-Compare (Algorithm 2)."""
    lib = _load()
    keep, a = _set(ss)
    out = np.zeros(4, np.uint64)
    n = lib.orc_lcp_compare(*a, a_idx, ha, b_idx, hb, _p(out, _u64p))
    return tuple(int(v) for v in out), int(n)


def lcp_merge2(ss, s1, h1, s2, h2):
    """(out, hout, comparisons) of binary LCP-merge (Algorithm 3)."""
    lib = _load()
    keep, a = _set(ss)
    s1, h1, s2, h2 = (_c(v, np.uint32) for v in (s1, h1, s2, h2))
    n = s1.shape[0] + s2.shape[0]
    out = np.empty(n, np.uint32)
    hout = np.empty(n, np.uint32)
    c = lib.orc_lcp_merge2(*a, _p(s1, _u32p), _p(h1, _u32p), s1.shape[0], _p(s2, _u32p),
                           _p(h2, _u32p), s2.shape[0], _p(out, _u32p), _p(hout, _u32p))
    return out, hout, int(c)


def lcp_mergek(ss, s, h, begin):
    """(out, hout, comparisons) of K-way LCP-merge (Algorithm 4); runs s[begin[k]:begin[k+1]]."""
    lib = _load()
    keep, a = _set(ss)
    s = _c(s, np.uint32)
    h = _c(h, np.uint32)
    begin = _c(begin, np.uint64)
    K = begin.shape[0] - 1
    out = np.empty(s.shape[0], np.uint32)
    hout = np.empty(s.shape[0], np.uint32)
    c = lib.orc_lcp_mergek(*a, _p(s, _u32p), _p(h, _u32p), _p(begin, _u64p), K,
                           _p(out, _u32p), _p(hout, _u32p))
    return out, hout, int(c)


def lcp_insertion(ss, s, hbar: int = 0):
    """(sorted s, lcp, comparisons) of LCP insertion sort (Algorithm 5)."""
    lib = _load()
    keep, a = _set(ss)
    s = _c(s, np.uint32).copy()
    h = np.empty(s.shape[0], np.uint32)
    c = lib.orc_lcp_insertion(*a, _p(s, _u32p), _p(h, _u32p), s.shape[0], hbar)
    return s, h, int(c)


def check_sorted(ss, perm, lcp):
    """(failures, first failing position): perm is a permutation, neighbours in
    order (ties by index), lcp[0] = 0 and lcp[i] the naive LCP, at every position."""
    lib = _load()
    keep, a = _set(ss)
    perm = _c(perm, np.uint32)
    lcp = _c(lcp, np.uint32)
    first = C.c_uint64()
    bad = lib.orc_check_sorted(*a, perm.shape[0], _p(perm, _u32p), _p(lcp, _u32p), C.byref(first))
    return int(bad), int(first.value)
