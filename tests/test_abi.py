"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/ss.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ss.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|uint64_t)\s+(ss_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("ss_sort", "ss_sort_ex", "ss_sort_host", "ss_sort_batch", "ss_merge", "ss_gather_keys",
                 "ss_splitters", "ss_classify", "ss_last_error_detail"):
        assert must in names


def test_library_builds_and_exports_all_symbols():
    from paper_1403_2056_gb300 import build
    so = build.build()
    lib = ctypes.CDLL(so)
    for name in _declared():
        assert hasattr(lib, name), name
    assert lib.ss_version() == 101


def test_binding_has_same_names():
    import paper_1403_2056_gb300 as P
    for name in _declared():
        if name in ("ss_last_error_detail", "ss_version", "ss_profile_enable", "ss_profile_reset",
                    "ss_profile_read", "ss_launch_count"):
            continue
        assert hasattr(P, name), name


def test_error_paths_without_gpu():
    """Argument errors are caught on the host before any CUDA call."""
    import paper_1403_2056_gb300 as P
    L = P.lib()
    assert L.ss_sort(None, None, 0, None, None, None) == 0          # n = 0 is a no-op
    assert L.ss_sort(None, None, 5, None, None, None) == -1         # NULL with n > 0
    assert L.ss_splitters(None, 0, 3, None, None) == -1
    buf = ctypes.create_string_buffer(256)
    assert L.ss_last_error_detail(buf, 256) > 0
    rb = (ctypes.c_uint32 * 3)(0, 5, 3)                             # decreasing run starts
    assert L.ss_merge(1, 1, None, 0, 1, 1, ctypes.cast(rb, ctypes.c_void_p), None, 2, 1, 1, None) == -1


def test_product_path_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_1403_2056_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", txt).replace("oracle array", ""), f


def test_tuning_ranges_checked_on_the_host():
    """Out-of-range tunings are refused before any device work."""
    import ctypes as C
    import paper_1403_2056_gb300 as P
    q = P.Request(1, 1, None, 0, 5, 1, 1, None)   # pointers are never dereferenced: the check fails first
    arr = (P.Request * 1)(q)
    # alphabets: unsorted, a zero byte, or a request that is not fixed-length (q is NUL-terminated)
    # max_depth outside [2, 8]; small_max not a power of two in [64, 2048]
    for bad in [(48, 0, 0), (16, 0, 0), (1 << 17, 0, 0), (0, 10, 0), (0, 0, 3), (0, 0, 0, 0x41434700),
                (0, 0, 0, 0x41474341), (0, 0, 0, 0x54474341), (0, 0, 0, 0, 1), (0, 0, 0, 0, 9),
                (0, 0, 0, 0, 0, 32), (0, 0, 0, 0, 0, 4096), (0, 0, 0, 0, 0, 1000)]:
        t = (P.Tuning * 1)(P.Tuning(*bad))
        rc = P.lib().ss_sort_batch_tuned(C.cast(arr, C.c_void_p), C.cast(t, C.c_void_p), 1, None)
        assert rc == -1, bad
        assert b"ss_sort_batch_tuned" in P._detail().encode()


def test_classifier_range_checked_on_the_host():
    """ss_classify_ex refuses an unknown classifier before any device work."""
    import paper_1403_2056_gb300 as P
    rc = P.lib().ss_classify_ex(None, 0, None, 3, 3, None, None, None, None)
    assert rc == -1
    assert "classifier" in P._detail()


def test_header_is_plain_c_and_cxx(tmp_path):
    """include/ss.h compiles as strict C99 and as C++ (a C ABI with no torch or
    CUDA types beyond an opaque stream pointer)."""
    import shutil
    import subprocess
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "use_header.c"
    src.write_text('#include "ss.h"\n'
                   "int main(void) { ss_tuning t = {0, 0, SS_CLASSIFIER_JUMP}; (void)t;\n"
                   "  ss_request q = {0}; (void)q; return SS_ERR_CANCELLED == -8 ? 0 : 1; }\n")
    for cc, args in (("gcc", ["-std=c99", "-pedantic", "-Werror", "-Wall"]), ("g++", ["-std=c++11", "-x", "c++"])):
        if shutil.which(cc) is None:
            continue
        subprocess.run([cc, *args, "-I", inc, "-c", str(src), "-o", str(tmp_path / f"o_{cc}.o")], check=True)


def test_host_buffer_arguments_checked_before_any_device_work():
    """ss_sort_host refuses host arrays of the wrong element size, shape or
    length in the binding, before the library is called."""
    import numpy as np
    import paper_1403_2056_gb300 as P
    chars = np.frombuffer(b"b\0a\0", np.uint8).copy()
    offs = np.array([0, 2], np.uint64)
    good = lambda: np.zeros(2, np.uint32)
    bad_cases = [
        (dict(perm_out=np.zeros(2, np.float32)), TypeError),
        (dict(lcp_out=np.zeros(1, np.uint32)), ValueError),
        (dict(offsets=np.array([0, 2], np.uint32)), TypeError),
        (dict(perm_out=np.zeros((2, 1), np.uint32)), ValueError),
        (dict(lengths=np.array([1], np.uint32)), ValueError),
    ]
    for change, exc in bad_cases:
        args = dict(chars=chars, offsets=offs, lengths=None, fixed_len=0, perm_out=good(), lcp_out=good())
        args.update(change)
        with pytest.raises(exc):
            P.ss_sort_host(**args)


def test_merge_run_tables_checked_in_the_binding():
    """ss_merge's host run tables are checked before any device buffer is
    looked at: K + 1 non-decreasing run starts and K index bases."""
    import paper_1403_2056_gb300 as P
    with pytest.raises(ValueError):
        P.ss_merge(1, 1, None, 0, 1, 1, [0, 5, 3], 1, 1)
    with pytest.raises(ValueError):
        P.ss_merge(1, 1, None, 0, 1, 1, [0, 2, 4], 1, 1, run_base=[0])
    with pytest.raises(ValueError):
        P.ss_merge_noalloc(1, 1, None, 0, 1, 1, [], 1, 1)
    # an unknown merge method is refused by the library before any device work
    with pytest.raises(P.SortError) as ei:
        P.ss_merge_ex(1, 1, None, 0, 1, 1, [0, 1, 2], 1, 1, method=7, stream=0)
    assert ei.value.status == -1 and "method" in ei.value.detail


def test_device_buffer_length_rule():
    """The binding's length rule for device tensors (checked on CPU tensors
    here; the GPU test calls the entry points with CUDA tensors)."""
    import torch
    import paper_1403_2056_gb300 as P
    P._need(torch.zeros(4), 4, "x")
    P._need(torch.zeros(4), None, "x")
    with pytest.raises(ValueError):
        P._need(torch.zeros(3), 4, "x")


def test_cache_arguments_checked_on_the_host():
    """A sort cache with only some of its arrays, a cache on an alphabet-
    compressed request, and ss_merge_cached without caches are refused before
    any device work (the pointers are never dereferenced)."""
    import ctypes as C
    import paper_1403_2056_gb300 as P
    q = P.Request(1, 1, None, 5, 5, 1, 1, None)   # fixed-length, 5 strings
    arr = (P.Request * 1)(q)
    for cache, tune in [((1, None, None), None), ((1, 1, None), None), ((None, None, 1), None),
                        ((1, 1, 1), (0, 0, 0, P.alphabet(b"ACGT")))]:
        carr = (P.SortCache * 1)(P.SortCache(*cache))
        tarr = None if tune is None else (P.Tuning * 1)(P.Tuning(*tune))
        rc = P.lib().ss_sort_batch_cached(C.cast(arr, C.c_void_p), None if tarr is None else C.cast(tarr, C.c_void_p),
                                          C.cast(carr, C.c_void_p), 1, None)
        assert rc == -1, cache
        assert "ss_sort_batch_cached" in P._detail()
    rb = (C.c_uint32 * 3)(0, 1, 2)
    rc = P.lib().ss_merge_cached(1, 1, None, 0, 1, 1, None, 1, 1, C.cast(rb, C.c_void_p), None, 2, 1, 1, None)
    assert rc == -1
    assert "cache" in P._detail()
