"""The sort server (continuous batching): every request's result is the same
alone and in the mix, whatever batches the server happened to form; the
memory budget admits requests without changing results; oversize requests are
refused at submit time."""
import threading
import time

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import gpu_sort, to_device

pytestmark = pytest.mark.gpu


def _sets(count, seed):
    rng = np.random.default_rng(seed)
    sets = []
    for r in range(count):
        n = int(np.exp(rng.uniform(np.log(10), np.log(200_000))))
        g = r % 4
        if g == 0:
            sets.append(W.random_lower(n, seed=5000 + r))
        elif g == 1:
            sets.append(W.url_like(n, seed=6000 + r))
        elif g == 2:
            sets.append(W.dna_windows(n, 20 * n + 100, 100, seed=7000 + r))
        else:
            sets.append(W.sinha_dna_like(n, seed=8000 + r))
    return sets


def _request(ss, torch):
    chars, offsets, lengths = to_device(ss)
    n = ss.n
    perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda:0")
    lcp = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda:0")
    status = torch.full((1,), -7, dtype=torch.int32, device="cuda:0")
    return dict(chars=chars, offsets=offsets, lengths=lengths, fixed_len=ss.fixed_len, n=n,
                perm_out=perm, lcp_out=lcp, status_out=status)


def _serve(sets, budget, workers, max_batch=0, jitter_ms=2.0, seed=0):
    import torch
    import paper_1403_2056_gb300 as P
    reqs = [_request(ss, torch) for ss in sets]
    torch.cuda.synchronize()
    rng = np.random.default_rng(seed)
    delays = rng.uniform(0, jitter_ms, len(reqs)) / 1e3
    tickets = [None] * len(reqs)
    with P.Server(budget, workers=workers, max_batch=max_batch) as srv:
        def producer():
            for k, q in enumerate(reqs):
                time.sleep(float(delays[k]))
                tickets[k] = srv.submit(q)
        th = threading.Thread(target=producer)
        th.start()
        th.join()
        results = [srv.wait(t) for t in tickets]
    torch.cuda.synchronize()
    return reqs, results


def _check_same_as_alone(sets, reqs, results):
    for ss, q, (status, times) in zip(sets, reqs, results):
        assert status == 0, ss.name
        assert int(q["status_out"].item()) == 0, ss.name
        assert times[0] <= times[1] <= times[2], (ss.name, times)
        want_perm, want_lcp = gpu_sort(ss)
        n = ss.n
        assert np.array_equal(q["perm_out"][:n].cpu().numpy().view(np.uint32), want_perm), ss.name
        assert np.array_equal(q["lcp_out"][:n].cpu().numpy().view(np.uint32), want_lcp), ss.name


def test_server_mix_equals_alone():
    """48 requests of 10..200,000 strings from four generators, submitted with
    random gaps to a 3-worker server: each result equals the request sorted
    alone, and the small ones equal the oracle."""
    sets = _sets(48, seed=11)
    reqs, results = _serve(sets, budget=8 << 30, workers=3)
    _check_same_as_alone(sets, reqs, results)
    for ss, q in zip(sets, reqs):
        if ss.n <= 20_000:
            want_perm, want_lcp = oracle.sort(ss)
            assert np.array_equal(q["perm_out"][:ss.n].cpu().numpy().view(np.uint32), want_perm), ss.name
            assert np.array_equal(q["lcp_out"][:ss.n].cpu().numpy().view(np.uint32), want_lcp), ss.name


def test_server_tight_budget_and_batch_limit():
    """A budget that admits the largest request only on its own, and batches of
    at most 3 requests: same results."""
    import paper_1403_2056_gb300 as P
    sets = _sets(24, seed=12)
    budget = max(P.ss_scratch_bytes(ss.n) for ss in sets)
    reqs, results = _serve(sets, budget=budget, workers=2, max_batch=3, jitter_ms=0.5, seed=1)
    _check_same_as_alone(sets, reqs, results)


def test_server_burst_batches_together():
    """A burst submitted with no gaps to a 1-worker server: later requests wait
    for the worker and then run together (their start times coincide)."""
    sets = _sets(16, seed=13)
    reqs, results = _serve(sets, budget=8 << 30, workers=1, jitter_ms=0.0)
    _check_same_as_alone(sets, reqs, results)
    starts = [t[1] for _, t in results]
    assert len(set(starts)) < len(starts)


def test_server_refuses_oversize_request():
    import torch
    import paper_1403_2056_gb300 as P
    ss = W.random_lower(50_000, seed=3)
    q = _request(ss, torch)
    with P.Server(P.ss_scratch_bytes(ss.n) - 1, workers=1) as srv:
        with pytest.raises(P.SortError) as e:
            srv.submit(q)
        assert e.value.status == -5


def test_server_host_requests_equal_sort_host():
    """Host-buffer requests (copies in, sort of runs + merge, copies out) on a
    2-worker server, several in flight: each equals ss_sort_host's result."""
    import torch
    import paper_1403_2056_gb300 as P
    sets = [W.url_like(150_000, seed=21), W.dna_windows(120_000, 2_400_100, 100, seed=22),
            W.random_lower(90_000, seed=23), W.url_like(60_000, seed=24)]
    with P.Server(8 << 30, workers=2) as srv:
        jobs = []
        for k, ss in enumerate(sets):
            hp = np.full(ss.n, 0xFFFFFFFF, np.uint32)
            hl = np.full(ss.n, 0xFFFFFFFF, np.uint32)
            runs = 1 + k % 3
            t = srv.submit_host(ss.chars, ss.offsets, None, ss.fixed_len, hp, hl, runs=runs)
            jobs.append((ss, runs, hp, hl, t))
        for ss, runs, hp, hl, t in jobs:
            status, _ = srv.wait(t)
            assert status == 0
            wp = np.full(ss.n, 0xFFFFFFFF, np.uint32)
            wl = np.full(ss.n, 0xFFFFFFFF, np.uint32)
            P.ss_sort_host(ss.chars, ss.offsets, None, ss.fixed_len, wp, wl, runs=runs)
            assert np.array_equal(hp, wp), ss.name
            assert np.array_equal(hl, wl), ss.name
            want_perm, want_lcp = oracle.sort(ss)
            assert np.array_equal(hp, want_perm), ss.name
            assert np.array_equal(hl, want_lcp), ss.name
