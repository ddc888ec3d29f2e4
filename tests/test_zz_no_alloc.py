"""ss_merge_noalloc: the merge for callers that cannot allocate (a process
whose device memory is owned by its own arena, a hard memory budget, or a
latency-critical path that must not call cudaMalloc/cudaFree).  Its output
must equal ss_merge's and the oracle's, bit for bit, on consecutive calls
that share the library's fixed scratch array.

The file name sorts last so that pytest collects it after every other test
file: it is a deployment variant outside the paper's method, and a run that
stops at its first failure (-x) has then already run all the other tests.
Nothing in it depends on what earlier tests left behind; it also passes run
alone in a fresh process."""
import numpy as np
import pytest

import workloads as W
from gpu_util import to_device

pytestmark = pytest.mark.gpu


def _runs(ss, K, seed):
    """K sorted runs of ss (index-contiguous, request-local indices) from ss_sort_batch."""
    import torch
    import paper_1403_2056_gb300 as P
    chars, offsets, lengths = to_device(ss)
    rng = np.random.default_rng(seed)
    cuts = np.sort(rng.integers(0, ss.n + 1, K - 1))
    rb = np.concatenate([[0], cuts, [ss.n]]).astype(np.uint32)
    rperm = torch.zeros(ss.n, dtype=torch.int32, device="cuda:0")
    rlcp = torch.zeros(ss.n, dtype=torch.int32, device="cuda:0")
    reqs = [dict(chars=chars, offsets=offsets[int(rb[k]):int(rb[k + 1])],
                 lengths=None if lengths is None else lengths[int(rb[k]):int(rb[k + 1])], fixed_len=ss.fixed_len,
                 n=int(rb[k + 1] - rb[k]), perm_out=rperm[int(rb[k]):int(rb[k + 1])],
                 lcp_out=rlcp[int(rb[k]):int(rb[k + 1])]) for k in range(K)]
    P.ss_sort_batch(reqs)
    return chars, offsets, lengths, rb, rperm, rlcp


def _merge_both(ss, K, seed):
    import torch
    import paper_1403_2056_gb300 as P
    chars, offsets, lengths, rb, rperm, rlcp = _runs(ss, K, seed)
    ref_p = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
    ref_l = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
    P.ss_merge(chars, offsets, lengths, ss.fixed_len, rperm, rlcp, rb, ref_p, ref_l, run_base=rb[:-1])
    out_p = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
    out_l = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
    P.ss_merge_noalloc(chars, offsets, lengths, ss.fixed_len, rperm, rlcp, rb, out_p, out_l, run_base=rb[:-1])
    torch.cuda.synchronize()
    return ref_p.cpu().numpy(), ref_l.cpu().numpy(), out_p.cpu().numpy(), out_l.cpu().numpy()


def test_noalloc_merge_equals_merge_on_two_calls_in_a_row():
    import oracle
    # first call: 5 runs (3 rounds through the fixed array); second: 3 runs of another set
    cases = [(W.url_like(300_000, seed=31), 5, 1), (W.dna_windows(200_000, 500_000, 100, seed=32), 3, 2)]
    for ss, K, seed in cases:
        ref_p, ref_l, out_p, out_l = _merge_both(ss, K, seed)
        assert np.array_equal(out_p, ref_p), ss.name
        assert np.array_equal(out_l, ref_l), ss.name
        want_p, want_l = oracle.sort(ss)
        assert np.array_equal(out_p.view(np.uint32), want_p), ss.name
        assert np.array_equal(out_l.view(np.uint32), want_l), ss.name


def test_noalloc_merge_rejects_beyond_limit():
    import torch
    import paper_1403_2056_gb300 as P
    ss = W.from_bytes_list([b"a", b"b"])
    chars, offsets, lengths = to_device(ss)
    # raw addresses: the binding cannot check their sizes, so the library's own
    # limit check is what refuses these (before any device work)
    buf = torch.zeros(2, dtype=torch.int32, device="cuda:0")
    b = buf.data_ptr()
    with pytest.raises(P.SortError) as ei:
        P.ss_merge_noalloc(chars, offsets.data_ptr(), None, 0, b, b, [0, 1, (1 << 20) + 1], b, b)
    assert ei.value.status == -5 and "limit" in ei.value.detail
    with pytest.raises(P.SortError) as ei:
        P.ss_merge_noalloc(chars, offsets.data_ptr(), None, 0, b, b, list(range(66)), b, b)
    assert ei.value.status == -5
