"""Python binding of libss_gb300.so, the GB300 string sample sorter.

Argument marshalling only: every function forwards torch tensors (device
memory, contiguous) or host numpy arrays to the C ABI declared in
include/ss.h and raises :class:`SortError` on a non-zero status.  There is no
CPU fallback: importing this module on a machine without the built library
raises immediately.

Names follow the C ABI: ss_sort, ss_sort_ex, ss_sort_host, ss_sort_batch,
ss_merge, ss_gather_keys, ss_splitters, ss_classify.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = [
    "SortError", "lib", "library_path",
    "ss_sort", "ss_sort_ex", "ss_sort_host", "ss_sort_batch", "ss_sort_batch_async", "ss_merge", "ss_merge_ex",
    "MERGE_PAIRWISE", "MERGE_LOSER_TREE",
    "ss_merge_noalloc", "ss_gather_keys", "ss_splitters", "ss_classify", "ss_classify_ex",
    "CLASSIFIER_UNROLL", "CLASSIFIER_EQUAL", "CLASSIFIER_JUMP", "alphabet",
    "profile_enable", "profile_reset", "profile_read", "launch_count", "ss_device_error", "ss_debug_copy_wait",
    "STATUS",
]

# classifiers (SS_CLASSIFIER_* of the C header)
CLASSIFIER_UNROLL, CLASSIFIER_EQUAL, CLASSIFIER_JUMP = 0, 1, 2
# merge methods (SS_MERGE_* of the C header)
MERGE_PAIRWISE, MERGE_LOSER_TREE = 0, 1

STATUS = {0: "SS_OK", -1: "SS_ERR_INVALID", -2: "SS_ERR_OOM", -3: "SS_ERR_CUDA", -4: "SS_ERR_TIMEOUT",
          -5: "SS_ERR_TOO_LARGE", -6: "SS_ERR_UNIMPLEMENTED", -7: "SS_ERR_INTERNAL", -8: "SS_ERR_CANCELLED"}


class SortError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__(f"{STATUS.get(status, status)}: {detail}")
        self.status = status
        self.detail = detail


def library_path() -> str:
    return _build.SO


_lib = None


def lib():
    """Load libss_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run `python -m paper_1403_2056_gb300.build` "
                          "(or __graft_entry__.build()) first; there is no CPU fallback")
    L = C.CDLL(path)
    vp, u32, u64, i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
    L.ss_sort.argtypes = [vp, vp, u32, vp, vp, vp]
    L.ss_sort_ex.argtypes = [vp, vp, vp, u32, u32, vp, vp, vp]
    L.ss_sort_host.argtypes = [vp, u64, vp, vp, u32, u32, u32, vp, vp, vp]
    L.ss_sort_batch.argtypes = [vp, u32, vp]
    L.ss_merge.argtypes = [vp, vp, vp, u32, vp, vp, vp, vp, u32, vp, vp, vp]
    L.ss_merge_noalloc.argtypes = [vp, vp, vp, u32, vp, vp, vp, vp, u32, vp, vp, vp]
    L.ss_merge_ex.argtypes = [vp, vp, vp, u32, vp, vp, vp, vp, u32, u32, vp, vp, vp]
    L.ss_gather_keys.argtypes = [vp, vp, vp, u32, u32, vp, vp, vp]
    L.ss_splitters.argtypes = [vp, u32, u32, vp, vp]
    L.ss_classify.argtypes = [vp, u32, vp, u32, vp, vp, vp, vp]
    L.ss_classify_ex.argtypes = [vp, u32, vp, u32, u32, vp, vp, vp, vp]
    L.ss_profile_enable.argtypes = [i32]
    L.ss_profile_read.argtypes = [vp, vp, vp, vp, i32]
    L.ss_launch_count.restype = u64
    L.ss_last_error_detail.argtypes = [C.c_char_p, C.c_size_t]
    L.ss_version.restype = i32
    L.ss_server_create.argtypes = [u64, u32, u32, C.POINTER(vp)]
    L.ss_server_submit.argtypes = [vp, vp, C.POINTER(u64)]
    L.ss_server_wait.argtypes = [vp, u64, C.POINTER(i32), C.POINTER(C.c_double)]
    L.ss_server_submit_host.argtypes = [vp, vp, C.POINTER(u64)]
    L.ss_sort_batch_tuned.argtypes = [vp, vp, u32, vp]
    L.ss_sort_batch_async.argtypes = [vp, vp, u32, vp]
    L.ss_sort_batch_cached.argtypes = [vp, vp, vp, u32, vp]
    L.ss_merge_cached.argtypes = [vp, vp, vp, u32, vp, vp, vp, vp, vp, vp, vp, u32, vp, vp, vp]
    L.ss_autotune.argtypes = [vp, u32, C.POINTER(Tuning), C.POINTER(C.c_double), vp]
    L.ss_server_destroy.argtypes = [vp]
    L.ss_server_cancel.argtypes = [vp, u64, C.POINTER(i32)]
    L.ss_debug_fail_allocs.argtypes = [u32, u32]
    L.ss_debug_copy_wait.argtypes = [u64, u32]
    L.ss_device_error.argtypes = [C.POINTER(i32)]
    L.ss_scratch_bytes.argtypes = [u32]
    L.ss_scratch_bytes.restype = u64
    for name in ("ss_sort", "ss_sort_ex", "ss_sort_host", "ss_sort_batch", "ss_merge", "ss_merge_ex", "ss_merge_noalloc",
                 "ss_gather_keys",
                 "ss_splitters", "ss_classify", "ss_classify_ex", "ss_profile_enable", "ss_profile_reset", "ss_profile_read",
                 "ss_server_create", "ss_server_submit", "ss_server_wait", "ss_server_destroy",
                 "ss_server_submit_host", "ss_sort_batch_tuned", "ss_sort_batch_async", "ss_sort_batch_cached",
                 "ss_merge_cached", "ss_autotune",
                 "ss_server_cancel",
                 "ss_debug_fail_allocs", "ss_debug_copy_wait", "ss_device_error"):
        getattr(L, name).restype = i32
    _lib = L
    return L


class HostRequest(C.Structure):
    _fields_ = [("chars", C.c_void_p), ("chars_len", C.c_uint64), ("offsets", C.c_void_p), ("lengths", C.c_void_p),
                ("fixed_len", C.c_uint32), ("n", C.c_uint32), ("runs", C.c_uint32), ("perm_out", C.c_void_p),
                ("lcp_out", C.c_void_p)]


class Tuning(C.Structure):
    _fields_ = [("child_target", C.c_uint32), ("min_step", C.c_uint32), ("classifier", C.c_uint32),
                ("alphabet", C.c_uint32), ("max_depth", C.c_uint32), ("small_max", C.c_uint32)]


def alphabet(symbols: bytes) -> int:
    """SS_ALPHABET of up to four bytes (sorted, the last repeated for fewer)."""
    b = sorted(set(symbols))
    if not 1 <= len(b) <= 4 or b[0] == 0:
        raise ValueError("an alphabet holds 1..4 non-zero bytes")
    b = b + [b[-1]] * (4 - len(b))
    return b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24)


class Request(C.Structure):
    """ss_request of the C ABI."""
    _fields_ = [("chars", C.c_void_p), ("offsets", C.c_void_p), ("lengths", C.c_void_p),
                ("fixed_len", C.c_uint32), ("n", C.c_uint32), ("perm_out", C.c_void_p),
                ("lcp_out", C.c_void_p), ("status_out", C.c_void_p)]


def _detail() -> str:
    buf = C.create_string_buffer(512)
    lib().ss_last_error_detail(buf, 512)
    return buf.value.decode(errors="replace")


def _check(rc: int):
    if rc != 0:
        raise SortError(rc, _detail())


def _ptr(t):
    """Device/host address of a torch tensor, numpy array or int (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return t.ctypes.data
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _need(t, min_len, what):
    """A device tensor must hold at least min_len elements: the kernels index
    it up to min_len - 1 and nothing on the device checks the bound."""
    if min_len is not None and t.numel() < min_len:
        raise ValueError(f"{what} holds {t.numel()} elements, needs {min_len}")


def _dev(t, dtype_name, what, min_len=None):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"{what} must be torch.{dtype_name}, got {t.dtype}")
    _need(t, min_len, what)
    return _ptr(t)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def ss_sort(chars, offsets, n, perm_out, lcp_out, stream=None):
    n = int(n)
    _check(lib().ss_sort(_dev(chars, "uint8", "chars"), _off(offsets, "offsets", n), n,
                         _dev(perm_out, "int32", "perm_out", n), _dev(lcp_out, "int32", "lcp_out", n),
                         _stream(stream)))


def ss_sort_ex(chars, offsets, lengths, fixed_len, n, perm_out, lcp_out, stream=None):
    n = int(n)
    _check(lib().ss_sort_ex(_dev(chars, "uint8", "chars"), _off(offsets, "offsets", n),
                            _dev(lengths, "int32", "lengths", n), int(fixed_len), n,
                            _dev(perm_out, "int32", "perm_out", n), _dev(lcp_out, "int32", "lcp_out", n),
                            _stream(stream)))


def _off(offsets, what="offsets", min_len=None):
    """A 64-bit device tensor (offsets, keys, splitters)."""
    if offsets is None or isinstance(offsets, int):
        return offsets
    if str(offsets.dtype) not in ("torch.int64", "torch.uint64"):
        raise TypeError(f"{what} must be a 64-bit integer tensor")
    if not offsets.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    _need(offsets, min_len, what)
    return _ptr(offsets)


def _host(a, itemsize, what, min_len=None):
    """Checks a host array (numpy or CPU tensor): integer elements of the given
    size, one dimension, at least min_len of them."""
    if a is None:
        return
    if isinstance(a, np.ndarray):
        ok_kind, size, length, on_host = a.dtype.kind in "iu", a.dtype.itemsize, a.size, True
        ndim = a.ndim
    else:
        ok_kind = not (a.dtype.is_floating_point or a.dtype.is_complex)
        size, length, on_host, ndim = a.element_size(), a.numel(), not a.is_cuda, a.dim()
    if not on_host:
        raise ValueError(f"{what} must be a host array")
    if not ok_kind or size != itemsize:
        raise TypeError(f"{what} must hold {8 * itemsize}-bit integers")
    if ndim != 1:
        raise ValueError(f"{what} must be one-dimensional")
    if min_len is not None and length < min_len:
        raise ValueError(f"{what} holds {length} elements, needs {min_len}")


def _check_host_request(chars, offsets, lengths, perm_out, lcp_out):
    n = int(offsets.shape[0])
    _host(chars, 1, "chars")
    _host(offsets, 8, "offsets")
    _host(lengths, 4, "lengths", n)
    _host(perm_out, 4, "perm_out", n)
    _host(lcp_out, 4, "lcp_out", n)
    return n


def ss_sort_host(chars, offsets, lengths, fixed_len, perm_out, lcp_out, runs=1, stream=None):
    """Host arrays (numpy, or pinned CPU tensors) in and out; the copies happen inside the call."""
    n = _check_host_request(chars, offsets, lengths, perm_out, lcp_out)
    nbytes = int(chars.nbytes) if isinstance(chars, np.ndarray) else int(chars.numel() * chars.element_size())
    _check(lib().ss_sort_host(_ptr(chars), nbytes, _ptr(offsets), _ptr(lengths), int(fixed_len), n, int(runs),
                              _ptr(perm_out), _ptr(lcp_out), _stream(stream)))


def ss_sort_batch(requests, stream=None):
    """requests: list of dicts with keys chars, offsets, lengths, fixed_len, n, perm_out, lcp_out, status_out."""
    arr = (Request * max(1, len(requests)))()
    for k, q in enumerate(requests):
        arr[k] = _request(q)
    _check(lib().ss_sort_batch(C.cast(arr, C.c_void_p), len(requests), _stream(stream)))


def _request(q):
    n = int(q["n"])
    return Request(_dev(q["chars"], "uint8", "chars"), _off(q["offsets"], "offsets", n),
                   _dev(q.get("lengths"), "int32", "lengths", n), int(q.get("fixed_len", 0)), n,
                   _dev(q["perm_out"], "int32", "perm_out", n), _dev(q["lcp_out"], "int32", "lcp_out", n),
                   _dev(q.get("status_out"), "int32", "status_out", 1))


def _tuned_args(requests, tunings):
    arr = (Request * max(1, len(requests)))()
    for k, q in enumerate(requests):
        arr[k] = _request(q)
    tarr = None
    if tunings is not None:
        tarr = (Tuning * max(1, len(requests)))()
        for k, t in enumerate(tunings):
            tarr[k] = Tuning(*[int(t[f]) if len(t) > f else 0 for f in range(6)])
    return arr, tarr


def ss_sort_batch_async(requests, tunings=None, stream=None):
    """As ss_sort_batch_tuned, but only queues the sort (levels launched from
    the device): outputs and each request's status_out are complete when the
    stream reaches this point.  The caller keeps the tensors alive until then."""
    arr, tarr = _tuned_args(requests, tunings)
    _check(lib().ss_sort_batch_async(C.cast(arr, C.c_void_p), None if tarr is None else C.cast(tarr, C.c_void_p),
                                      len(requests), _stream(stream)))


def ss_sort_batch_tuned(requests, tunings=None, stream=None):
    """As ss_sort_batch, with one (child_target, min_step[, classifier[, alphabet]]) tuple per request
    (0: default; alphabet from alphabet(b"ACGT") for fixed-length requests over at most four bytes)."""
    arr = (Request * max(1, len(requests)))()
    for k, q in enumerate(requests):
        arr[k] = _request(q)
    tarr = None
    if tunings is not None:
        tarr = (Tuning * max(1, len(requests)))()
        for k, t in enumerate(tunings):
            tarr[k] = Tuning(*[int(t[f]) if len(t) > f else 0 for f in range(6)])
    _check(lib().ss_sort_batch_tuned(C.cast(arr, C.c_void_p), None if tarr is None else C.cast(tarr, C.c_void_p),
                                      len(requests), _stream(stream)))


def ss_autotune(q, sample_n: int = 0, stream=None):
    """((child_target, min_step, classifier, alphabet, max_depth, small_max), ms): the tuning fastest
    on the first sample_n strings of request q (a tuple in ss_tuning's field order)."""
    t = Tuning()
    ms = C.c_double()
    _check(lib().ss_autotune(C.byref(_request(q)), int(sample_n), C.byref(t), C.byref(ms), _stream(stream)))
    return (t.child_target, t.min_step, t.classifier, t.alphabet, t.max_depth, t.small_max), ms.value


def ss_scratch_bytes(n: int) -> int:
    return int(lib().ss_scratch_bytes(int(n)))


def ss_server_create(budget_bytes: int, workers: int = 2, max_batch: int = 0):
    h = C.c_void_p()
    _check(lib().ss_server_create(int(budget_bytes), int(workers), int(max_batch), C.byref(h)))
    return h


def ss_server_submit(server, q) -> int:
    t = C.c_uint64()
    _check(lib().ss_server_submit(server, C.byref(_request(q)), C.byref(t)))
    return t.value


def ss_server_submit_host(server, chars, offsets, lengths, fixed_len, perm_out, lcp_out, runs=1) -> int:
    """Host arrays (numpy, or pinned CPU tensors), as for ss_sort_host."""
    n = _check_host_request(chars, offsets, lengths, perm_out, lcp_out)
    nbytes = int(chars.nbytes) if isinstance(chars, np.ndarray) else int(chars.numel() * chars.element_size())
    q = HostRequest(_ptr(chars), nbytes, _ptr(offsets), _ptr(lengths), int(fixed_len), n, int(runs), _ptr(perm_out),
                    _ptr(lcp_out))
    t = C.c_uint64()
    _check(lib().ss_server_submit_host(server, C.byref(q), C.byref(t)))
    return t.value


def ss_server_wait(server, ticket: int):
    st = C.c_int32()
    tm = (C.c_double * 3)()
    _check(lib().ss_server_wait(server, int(ticket), C.byref(st), tm))
    return int(st.value), (tm[0], tm[1], tm[2])


def ss_server_cancel(server, ticket: int) -> bool:
    """True if the request was still queued and is withdrawn (its wait reports
    SS_ERR_CANCELLED); False if a worker already took it."""
    c = C.c_int32()
    _check(lib().ss_server_cancel(server, int(ticket), C.byref(c)))
    return bool(c.value)


def ss_server_destroy(server):
    _check(lib().ss_server_destroy(server))


def ss_debug_fail_allocs(skip: int, count: int):
    """Host-side fault injection for tests: after `skip` successful scratch
    allocations, the next `count` fail as an exhausted pool would (0: off)."""
    _check(lib().ss_debug_fail_allocs(int(skip), int(count)))


def ss_device_error() -> int:
    """The first device-side failure (ss_status code) of any asynchronous sort
    since the last call, 0 if none; synchronize the sorts' streams first."""
    v = C.c_int32()
    _check(lib().ss_device_error(C.byref(v)))
    return int(v.value)


def ss_debug_copy_wait(budget_cycles: int, withhold: bool):
    """Test hook of the timeout path (see include/ss.h): wait budget of the
    distribution step's bulk copies, and whether the copies are withheld."""
    _check(lib().ss_debug_copy_wait(int(budget_cycles), 1 if withhold else 0))


class Server:
    """Continuous-batching sort server (ss_server_* of the C ABI).  submit()
    queues a request dict (keys as for ss_sort_batch) and returns its ticket;
    wait(ticket) blocks until it is done and returns (status, (t_submit,
    t_start, t_done)) in ms on the server's clock.  The caller keeps the
    request's tensors alive until wait() has returned."""

    def __init__(self, budget_bytes: int, workers: int = 2, max_batch: int = 0):
        self._h = ss_server_create(budget_bytes, workers, max_batch)
        self._keep = {}

    def submit(self, q) -> int:
        t = ss_server_submit(self._h, q)
        self._keep[t] = q
        return t

    def submit_host(self, chars, offsets, lengths, fixed_len, perm_out, lcp_out, runs=1) -> int:
        t = ss_server_submit_host(self._h, chars, offsets, lengths, fixed_len, perm_out, lcp_out, runs)
        self._keep[t] = (chars, offsets, lengths, perm_out, lcp_out)
        return t

    def wait(self, ticket: int):
        r = ss_server_wait(self._h, ticket)
        self._keep.pop(ticket, None)
        return r

    def cancel(self, ticket: int) -> bool:
        return ss_server_cancel(self._h, ticket)

    def close(self):
        if self._h:
            ss_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _merge_args(chars, offsets, lengths, fixed_len, run_perm, run_lcp, run_begin, perm_out, lcp_out, run_base):
    """Marshals the arguments of ss_merge / ss_merge_noalloc.  Every device
    buffer must hold what the runs index: run_perm, run_lcp, perm_out and
    lcp_out run_begin[K] entries, offsets (and lengths) one per string index
    the runs name (run_base[k] + run k's length, or run_begin[K] without
    bases); run_base has K entries."""
    rb = np.ascontiguousarray(np.asarray(run_begin, dtype=np.uint32))
    if rb.ndim != 1 or rb.shape[0] < 1:
        raise ValueError("run_begin must list K + 1 run starts")
    K = rb.shape[0] - 1
    if np.any(rb[1:] < rb[:-1]):
        raise ValueError("run_begin must be non-decreasing")
    total = int(rb[-1]) if K else 0
    base = None
    strings = total
    if run_base is not None:
        base = np.ascontiguousarray(np.asarray(run_base, dtype=np.uint32))
        if base.ndim != 1 or base.shape[0] < K:
            raise ValueError(f"run_base holds {base.size} entries, needs {K}")
        sizes = rb[1:].astype(np.int64) - rb[:-1].astype(np.int64)
        strings = int((base[:K].astype(np.int64) + sizes).max()) if K else 0
    args = (_dev(chars, "uint8", "chars"), _off(offsets, "offsets", strings),
            _dev(lengths, "int32", "lengths", strings), int(fixed_len),
            _dev(run_perm, "int32", "run_perm", total), _dev(run_lcp, "int32", "run_lcp", total),
            rb.ctypes.data, None if base is None else base.ctypes.data, K,
            _dev(perm_out, "int32", "perm_out", total), _dev(lcp_out, "int32", "lcp_out", total))
    return args, (rb, base)


def ss_merge(chars, offsets, lengths, fixed_len, run_perm, run_lcp, run_begin, perm_out, lcp_out,
             run_base=None, stream=None):
    args, keep = _merge_args(chars, offsets, lengths, fixed_len, run_perm, run_lcp, run_begin, perm_out, lcp_out,
                             run_base)
    _check(lib().ss_merge(*args, _stream(stream)))
    del keep


def ss_merge_ex(chars, offsets, lengths, fixed_len, run_perm, run_lcp, run_begin, perm_out, lcp_out,
                run_base=None, method=MERGE_PAIRWISE, stream=None):
    """ss_merge with the merge method chosen (MERGE_PAIRWISE or MERGE_LOSER_TREE)."""
    args, keep = _merge_args(chars, offsets, lengths, fixed_len, run_perm, run_lcp, run_begin, perm_out, lcp_out,
                             run_base)
    _check(lib().ss_merge_ex(*args[:9], int(method), *args[9:], _stream(stream)))
    del keep


class SortCache(C.Structure):
    _fields_ = [("off_out", C.c_void_p), ("ck_out", C.c_void_p), ("ckd_out", C.c_void_p)]


def ss_sort_batch_cached(requests, caches, tunings=None, stream=None):
    """ss_sort_batch_tuned that also writes, per request, the caches a later
    ss_merge_cached reads: caches[k] = (off_out int64[n], ck_out int64[n],
    ckd_out int32[n]) device tensors, or None."""
    arr, tarr = _tuned_args(requests, tunings)
    carr = (SortCache * max(1, len(requests)))()
    for k, q in enumerate(requests):
        c = caches[k] if caches is not None else None
        if c is not None:
            n = int(q["n"])
            carr[k] = SortCache(_dev(c[0], "int64", "off_out", n), _dev(c[1], "int64", "ck_out", n),
                                _dev(c[2], "int32", "ckd_out", n))
    _check(lib().ss_sort_batch_cached(C.cast(arr, C.c_void_p), None if tarr is None else C.cast(tarr, C.c_void_p),
                                      C.cast(carr, C.c_void_p), len(requests), _stream(stream)))


def ss_merge_cached(chars, offsets, lengths, fixed_len, run_perm, run_lcp, run_off, run_ck, run_ckd, run_begin,
                    perm_out, lcp_out, run_base=None, stream=None):
    """ss_merge of runs sorted by ss_sort_batch_cached, from their caches (laid out as run_perm)."""
    args, keep = _merge_args(chars, offsets, lengths, fixed_len, run_perm, run_lcp, run_begin, perm_out, lcp_out,
                             run_base)
    total = int(np.asarray(run_begin, dtype=np.uint32)[-1])
    cache = (_dev(run_off, "int64", "run_off", total), _dev(run_ck, "int64", "run_ck", total),
             _dev(run_ckd, "int32", "run_ckd", total))
    _check(lib().ss_merge_cached(*args[:6], *cache, *args[6:], _stream(stream)))
    del keep


def ss_merge_noalloc(chars, offsets, lengths, fixed_len, run_perm, run_lcp, run_begin, perm_out, lcp_out,
                     run_base=None, stream=None):
    """ss_merge without allocation (fixed 8 MiB device array; <= 1,048,576 strings, <= 64 runs).
    Only queues work on the stream: synchronize before reading the outputs."""
    args, keep = _merge_args(chars, offsets, lengths, fixed_len, run_perm, run_lcp, run_begin, perm_out, lcp_out,
                             run_base)
    _check(lib().ss_merge_noalloc(*args, _stream(stream)))
    del keep


def ss_gather_keys(chars, offsets, lengths, fixed_len, n, depth, keys_out, stream=None):
    n = int(n)
    _check(lib().ss_gather_keys(_dev(chars, "uint8", "chars"), _off(offsets, "offsets", n),
                                _dev(lengths, "int32", "lengths", n), int(fixed_len), n,
                                _dev(depth, "int32", "depth", n), _off(keys_out, "keys_out", n), _stream(stream)))


def ss_splitters(sample, a, d, x_out, stream=None):
    a, d = int(a), int(d)
    v = (1 << d) - 1 if 0 <= d < 32 else None
    _check(lib().ss_splitters(_off(sample, "sample", a), a, d, _off(x_out, "x_out", v), _stream(stream)))


def _classify_args(keys, n, x, d, bucket_out, bucket_begin_out, order_out):
    n, d = int(n), int(d)
    v = (1 << d) - 1 if 0 <= d < 32 else None
    return (_off(keys, "keys", n), n, _off(x, "x", v), d), (
        _dev(bucket_out, "int16", "bucket_out", n),
        _dev(bucket_begin_out, "int32", "bucket_begin_out", None if v is None else 2 * v + 2),
        _dev(order_out, "int32", "order_out", n))


def ss_classify(keys, n, x, d, bucket_out, bucket_begin_out, order_out, stream=None):
    head, outs = _classify_args(keys, n, x, d, bucket_out, bucket_begin_out, order_out)
    _check(lib().ss_classify(*head, *outs, _stream(stream)))


def ss_classify_ex(keys, n, x, d, classifier, bucket_out, bucket_begin_out, order_out, stream=None):
    head, outs = _classify_args(keys, n, x, d, bucket_out, bucket_begin_out, order_out)
    _check(lib().ss_classify_ex(*head, int(classifier), *outs, _stream(stream)))


def profile_enable(on: bool = True):
    _check(lib().ss_profile_enable(1 if on else 0))


def profile_reset():
    _check(lib().ss_profile_reset())


def profile_read(cap: int = 64):
    """{kernel name: (launches, total ms, units)} of the library's own launches since the last reset."""
    names = C.create_string_buffer(48 * cap)
    launches = (C.c_uint64 * cap)()
    ms = (C.c_double * cap)()
    units = (C.c_uint64 * cap)()
    k = lib().ss_profile_read(names, launches, ms, units, cap)
    out = {}
    for i in range(min(k, cap)):
        nm = names.raw[48 * i: 48 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (int(launches[i]), float(ms[i]), int(units[i]))
    return out


def launch_count() -> int:
    return int(lib().ss_launch_count())
