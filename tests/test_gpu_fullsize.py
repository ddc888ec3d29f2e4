"""GPU results at the workloads' full sizes, checked at every position against
the definitions (the oracle's any-size checker: permutation, neighbours in
order with ties by index, naive LCP), plus a batch of mixed requests checked
bit for bit against the oracle's own sort."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import gpu_sort, to_device

pytestmark = pytest.mark.gpu


def _assert_sorted(ss, perm, lcp):
    bad, first = oracle.check_sorted(ss, perm, lcp)
    assert bad == 0, f"{ss.name}: {bad} failing positions, first at {first}"


def test_url_like_10m_sort_and_runs_merge():
    """URL-like set, n = 10,000,000 (the benchmark workload): one ss_sort, and
    4 runs by ss_sort_batch + ss_merge, which must give the same arrays."""
    import torch
    import paper_1403_2056_gb300 as P
    ss = W.url_like(10_000_000, seed=2)
    chars, offsets, _ = to_device(ss)
    perm, lcp = gpu_sort(ss, chars, offsets, None)
    _assert_sorted(ss, perm, lcp)
    n, K = ss.n, 4
    rb = np.array([n * k // K for k in range(K + 1)], np.uint32)
    rperm = torch.empty(n, dtype=torch.int32, device="cuda:0")
    rlcp = torch.empty(n, dtype=torch.int32, device="cuda:0")
    reqs = [dict(chars=chars, offsets=offsets[int(rb[k]):int(rb[k + 1])], lengths=None, fixed_len=0,
                 n=int(rb[k + 1] - rb[k]), perm_out=rperm[int(rb[k]):int(rb[k + 1])],
                 lcp_out=rlcp[int(rb[k]):int(rb[k + 1])]) for k in range(K)]
    P.ss_sort_batch(reqs)
    mp = torch.empty(n, dtype=torch.int32, device="cuda:0")
    ml = torch.empty(n, dtype=torch.int32, device="cuda:0")
    P.ss_merge(chars, offsets, None, 0, rperm, rlcp, rb, mp, ml, run_base=rb[:-1])
    torch.cuda.synchronize()
    assert np.array_equal(mp.cpu().numpy().view(np.uint32), perm)
    assert np.array_equal(ml.cpu().numpy().view(np.uint32), lcp)
    # the other classifiers give the same arrays at full size
    for cls in (1, 2):
        cp = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
        cl = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
        P.ss_sort_batch_tuned([dict(chars=chars, offsets=offsets, lengths=None, fixed_len=0, n=n, perm_out=cp,
                                    lcp_out=cl)], [(0, 0, cls)])
        torch.cuda.synchronize()
        assert np.array_equal(cp.cpu().numpy().view(np.uint32), perm), cls
        assert np.array_equal(cl.cpu().numpy().view(np.uint32), lcp), cls


def test_dna_windows_20m():
    """DNA-like windows: 400,000,000-byte text, n = 20,000,000 windows of 100 bytes."""
    ss = W.dna_windows(n=20_000_000, text_len=400_000_000, window=100, seed=3)
    perm, lcp = gpu_sort(ss)
    _assert_sorted(ss, perm, lcp)


def test_no_lcp_64m():
    """n = 64 Mi strings of 16 bytes U[1,255]: near-zero LCPs."""
    ss = W.no_lcp(n=64 * 1024 * 1024, seed=5)
    perm, lcp = gpu_sort(ss)
    _assert_sorted(ss, perm, lcp)


def test_batch_of_mixed_requests():
    """Requests of log-uniform sizes 1,000..100,000 from the three generators
    (a reduced form of the batched configuration), each checked exactly."""
    import torch
    import paper_1403_2056_gb300 as P
    rng = np.random.default_rng(4)
    sets = []
    for r in range(192):
        n = int(np.exp(rng.uniform(np.log(1e3), np.log(1e5))))
        g = r % 3
        if g == 0:
            sets.append(W.random_lower(n, seed=1000 + r))
        elif g == 1:
            sets.append(W.url_like(n, seed=2000 + r))
        else:
            sets.append(W.dna_windows(n, 20 * n, 100, seed=3000 + r))
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


def test_dna_windows_20m_alphabet_compressed():
    """The same 20,000,000 DNA windows with alphabet compression (2-bit codes,
    32 characters per key): every position checked, and the arrays equal the
    byte-key sort's."""
    import torch
    import paper_1403_2056_gb300 as P
    ss = W.dna_windows(n=20_000_000, text_len=400_000_000, window=100, seed=3)
    chars, offsets, _ = to_device(ss)
    perm, lcp = gpu_sort(ss, chars, offsets, None)
    cp = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
    cl = torch.full((ss.n,), -1, dtype=torch.int32, device="cuda:0")
    P.ss_sort_batch_tuned([dict(chars=chars, offsets=offsets, lengths=None, fixed_len=100, n=ss.n, perm_out=cp,
                                lcp_out=cl)], [(0, 0, 0, P.alphabet(b"ACGT"))])
    torch.cuda.synchronize()
    cperm, clcp = cp.cpu().numpy().view(np.uint32), cl.cpu().numpy().view(np.uint32)
    _assert_sorted(ss, cperm, clcp)
    assert np.array_equal(cperm, perm) and np.array_equal(clcp, lcp)
