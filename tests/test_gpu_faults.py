"""Failure handling without a GPU fault: scratch-allocation failures injected
on the host (ss_debug_fail_allocs) make each entry point return SS_ERR_OOM
and leave the library usable; the server reports them per request and
withdraws queued requests on cancel.  Nothing here faults, traps or hangs
the device."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import to_device

pytestmark = pytest.mark.gpu

OOM, CANCELLED = -2, -8


def _outs(torch, n):
    return (torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda:0"),
            torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda:0"))


def _same(ss, perm, lcp):
    want_perm, want_lcp = oracle.sort(ss)
    return (np.array_equal(perm[:ss.n].cpu().numpy().view(np.uint32), want_perm)
            and np.array_equal(lcp[:ss.n].cpu().numpy().view(np.uint32), want_lcp))


def _expect_oom(fn):
    import paper_1403_2056_gb300 as P
    with pytest.raises(P.SortError) as e:
        fn()
    assert e.value.status == OOM
    P.ss_debug_fail_allocs(0, 0)


def test_injected_allocation_failures_then_recovery():
    import torch
    import paper_1403_2056_gb300 as P
    ss = W.url_like(120_000, seed=61)
    chars, offsets, _ = to_device(ss)
    perm, lcp = _outs(torch, ss.n)
    try:
        # one sort: its single scratch allocation fails
        P.ss_debug_fail_allocs(0, 1)
        _expect_oom(lambda: P.ss_sort(chars, offsets, ss.n, perm, lcp))
        P.ss_sort(chars, offsets, ss.n, perm, lcp)
        torch.cuda.synchronize()
        assert _same(ss, perm, lcp)
        # host buffers with 4 runs: the copy buffers, the sort of the runs and the merge fail in turn
        for skip in range(3):
            hp = np.full(ss.n, 0xFFFFFFFF, np.uint32)
            hl = np.full(ss.n, 0xFFFFFFFF, np.uint32)
            P.ss_debug_fail_allocs(skip, 1)
            _expect_oom(lambda: P.ss_sort_host(ss.chars, ss.offsets, None, 0, hp, hl, runs=4))
            P.ss_sort_host(ss.chars, ss.offsets, None, 0, hp, hl, runs=4)
            want_perm, want_lcp = oracle.sort(ss)
            assert np.array_equal(hp, want_perm) and np.array_equal(hl, want_lcp), skip
        # a batch
        perm2, lcp2 = _outs(torch, ss.n)
        q = dict(chars=chars, offsets=offsets, lengths=None, fixed_len=0, n=ss.n, perm_out=perm2, lcp_out=lcp2)
        P.ss_debug_fail_allocs(0, 1)
        _expect_oom(lambda: P.ss_sort_batch([q]))
        P.ss_sort_batch([q])
        torch.cuda.synchronize()
        assert _same(ss, perm2, lcp2)
    finally:
        P.ss_debug_fail_allocs(0, 0)


def test_server_reports_allocation_failure_per_request():
    import torch
    import paper_1403_2056_gb300 as P
    ss = W.random_lower(50_000, seed=62)
    chars, offsets, _ = to_device(ss)
    perm, lcp = _outs(torch, ss.n)
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda:0")
    q = dict(chars=chars, offsets=offsets, lengths=None, fixed_len=0, n=ss.n, perm_out=perm, lcp_out=lcp,
             status_out=status)
    try:
        with P.Server(8 << 30, workers=1) as srv:
            P.ss_debug_fail_allocs(0, 1)
            st, _ = srv.wait(srv.submit(q))
            assert st == OOM
            P.ss_debug_fail_allocs(0, 0)
            st, _ = srv.wait(srv.submit(q))
            assert st == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert _same(ss, perm, lcp)
    finally:
        P.ss_debug_fail_allocs(0, 0)


def test_server_cancel_withdraws_queued_requests():
    """A 1-worker server taking one request at a time: behind a 20 M-string
    request the small ones are still queued, so cancelling them withdraws them
    (outputs untouched, status SS_ERR_CANCELLED); the others finish."""
    import torch
    import paper_1403_2056_gb300 as P
    big = W.dna_windows(n=20_000_000, text_len=400_000_000, window=100, seed=63)
    bc, bo, _ = to_device(big)
    bperm, blcp = _outs(torch, big.n)
    small = [W.url_like(30_000, seed=64 + k) for k in range(5)]
    reqs = []
    for ss in small:
        c, o, _ = to_device(ss)
        p, l = _outs(torch, ss.n)
        reqs.append((ss, dict(chars=c, offsets=o, lengths=None, fixed_len=0, n=ss.n, perm_out=p, lcp_out=l)))
    torch.cuda.synchronize()
    with P.Server(64 << 30, workers=1, max_batch=1) as srv:
        tb = srv.submit(dict(chars=bc, offsets=bo, lengths=None, fixed_len=big.fixed_len, n=big.n,
                             perm_out=bperm, lcp_out=blcp))
        tickets = [srv.submit(q) for _, q in reqs]
        cancelled = {k: srv.cancel(tickets[k]) for k in (1, 3)}
        with pytest.raises(P.SortError):
            srv.cancel(10 ** 9)   # unknown ticket
        assert srv.wait(tb)[0] == 0
        results = [srv.wait(t)[0] for t in tickets]
    torch.cuda.synchronize()
    assert any(cancelled.values())
    for k, (ss, q) in enumerate(reqs):
        if cancelled.get(k):
            assert results[k] == CANCELLED
            assert int((q["perm_out"] != -1).sum().item()) == 0
        else:
            assert results[k] == 0
            assert _same(ss, q["perm_out"], q["lcp_out"])


def test_undersized_device_buffers_refused_by_the_binding():
    """A device tensor shorter than what the call indexes is refused in the
    binding (ValueError) before the library runs any kernel on it; the
    library keeps working afterwards."""
    import torch
    import paper_1403_2056_gb300 as P
    ss = W.random_lower(5_000, seed=67)
    chars, offsets, _ = to_device(ss)
    n = ss.n
    perm, lcp = _outs(torch, n)
    short = torch.zeros(n - 1, dtype=torch.int32, device="cuda:0")
    with pytest.raises(ValueError):
        P.ss_sort(chars, offsets, n, short, lcp)
    with pytest.raises(ValueError):
        P.ss_sort(chars, offsets, n, perm, short)
    with pytest.raises(ValueError):
        P.ss_sort(chars, offsets[: n - 1], n, perm, lcp)
    with pytest.raises(ValueError):
        P.ss_sort_batch([dict(chars=chars, offsets=offsets, n=n, perm_out=short, lcp_out=lcp)])
    depth = torch.zeros(n, dtype=torch.int32, device="cuda:0")
    keys = torch.zeros(n - 1, dtype=torch.int64, device="cuda:0")
    with pytest.raises(ValueError):
        P.ss_gather_keys(chars, offsets, None, 0, n, depth, keys)
    # merge: runs index up to run_begin[K]; offsets must cover run_base[k] + run length
    rb = [0, n // 2, n]
    with pytest.raises(ValueError):
        P.ss_merge(chars, offsets, None, 0, perm, lcp, rb, short, lcp, run_base=[0, n // 2])
    with pytest.raises(ValueError):
        P.ss_merge(chars, offsets, None, 0, perm, lcp, rb, perm, lcp, run_base=[0, n])
    with pytest.raises(ValueError):
        P.ss_merge(chars, offsets, None, 0, perm, lcp, rb, perm, lcp, run_base=[0])
    P.ss_sort(chars, offsets, n, perm, lcp)
    torch.cuda.synchronize()
    assert _same(ss, perm, lcp)


def test_bounded_copy_wait_runs_out_and_reports_timeout():
    """The distribution step's waits for its bulk copies are bounded: with the
    copies withheld (a flag nothing sets, as the test hook arranges) and a
    short budget, every wait runs out and the sort stops after that level.
    ss_sort_batch (levels driven from the host) returns SS_ERR_TIMEOUT and
    writes it to the request's status; ss_sort_batch_async (levels driven from
    the device) writes it to the status and ss_device_error reports it.  The
    library sorts correctly once the hook is off."""
    import torch
    import paper_1403_2056_gb300 as P
    TIMEOUT = -4
    ss = W.url_like(150_000, seed=71)
    chars, offsets, _ = to_device(ss)
    perm, lcp = _outs(torch, ss.n)
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda:0")
    req = dict(chars=chars, offsets=offsets, n=ss.n, perm_out=perm, lcp_out=lcp, status_out=status)
    P.ss_device_error()   # clear
    try:
        P.ss_debug_copy_wait(200_000, True)
        P.ss_sort_batch_async([req])
        torch.cuda.synchronize()
        assert int(status.item()) == TIMEOUT
        assert P.ss_device_error() == TIMEOUT
        assert P.ss_device_error() == 0   # read and cleared
        status.fill_(99)
        with pytest.raises(P.SortError) as e:
            P.ss_sort_batch([req])
        assert e.value.status == TIMEOUT
        torch.cuda.synchronize()
        assert int(status.item()) == TIMEOUT
    finally:
        P.ss_debug_copy_wait(0, False)
    for fn in (P.ss_sort_batch, P.ss_sort_batch_async):
        status.fill_(99)
        perm.fill_(-1)
        fn([req])
        torch.cuda.synchronize()
        assert int(status.item()) == 0 and P.ss_device_error() == 0
        assert _same(ss, perm, lcp)
