#!/usr/bin/env python
"""Throughput benchmark of the GB300 string sample sorter.

One step is one pass of the whole hot path over the URL-like workload
(n = 10,000,000 strings, seed 2): the set is cut into K = 4 index-contiguous
runs, ss_sort_batch_cached sorts the runs together (key gathers, splitter
trees, classification, histograms, prefix sums, scatter, recursion, base
case, LCP output, and each position's string offset and distinguishing
characters), then ss_merge_cached LCP-merges the runs from those into the
final permutation and LCP array.  The result is identical to one ss_sort of
the whole set.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (plain qsort + naive LCP, one thread)
on a bounded sample of the same workload instead.

With N > 1 (torchrun) every rank sorts its own replica of the workload:
the sort does not shard, there is no collective on the data path; the
barrier and the max over ranks only frame the timing.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "strings/s and D-GB/s vs HBM roofline (bit-exact); batched p50/p99 vs plain"

# Algorithmic bytes per unit of each kernel (unit = string, counter or record):
# the minimal traffic of the step the kernel performs, as the hot-path table
# lays out its inputs and outputs, independent of cache behaviour and of what
# this implementation carries beside it (CARRIED_BYTES_PER_UNIT).
BYTES_PER_UNIT = {
    # a1: offset read, 8-byte key gathered, key + string index written
    "init": 8 + 8 + 8 + 4,
    # a3: key read, bucket id (u16) written
    "classify": 8 + 2,
    # a6: bucket id read; string index (u32) and next key (u64) read and written
    "scatter": 2 + 4 + 8 + 4 + 8,
    # a8: index + key read, perm + lcp written
    "base_warp": 4 + 8 + 4 + 4,
    "base_c1": 4 + 8 + 4 + 4,
    "base_c2": 4 + 8 + 4 + 4,
    "base_c3": 4 + 8 + 4 + 4,
    # a9: two perm reads, two key gathers, lcp write
    "boundary": 4 + 4 + 8 + 8 + 4,
    # a10: per output of a merge round, (index, lcp) read and written
    "merge_round": 4 + 4 + 4 + 4,
    "merge_kway": 4 + 4 + 4 + 4,
    "copy_run": 16,
    "scan_reduce": 4,
    "scan_down": 8,
    "buckets": 8,
}
# Bytes per unit that this implementation moves beyond the table's layout by
# design (reported beside the roofline, never inside it): the scatter carries
# each string's 8-byte offset with its index (read and written) so that a
# later key gather is one random read instead of two.
CARRIED_BYTES_PER_UNIT = {"scatter": 8 + 8}


L2_BYTES = 129 * 1024 * 1024   # GB300 L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="url_like", choices=sorted(WORKLOADS),
                    help="the step's string set (default: the URL-like configuration)")
    ap.add_argument("--n", type=int, default=0, help="strings (0: the workload's configuration size)")
    ap.add_argument("--runs", type=int, default=4)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the DNA 20M and no-LCP 64Mi sorts")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-plain measurement")
    ap.add_argument("--batched-requests", type=int, default=4096)
    ap.add_argument("--no-serving", action="store_true", help="skip the served-vs-plain measurement")
    ap.add_argument("--e2e-workers", type=int, default=4, help="server workers for the end-to-end stream")
    ap.add_argument("--e2e-inflight", type=int, default=6, help="host-request steps in flight end to end")
    ap.add_argument("--e2e-steps", type=int, default=0, help="steps of the end-to-end stream (0: max(30, --steps))")
    ap.add_argument("--serving-requests", type=int, default=20000)
    ap.add_argument("--capture", action="store_true",
                    help="for counter captures: only the warm-up steps, the timed steps and the profiled steps run "
                         "(no sort-only calls), so every launch belongs to one of max(W, 3) + 2 K identical steps")
    return ap.parse_args()


def other_workloads(P, torch, dev, stream, peak):
    """One ss_sort of each other full-size workload (device-resident inputs):
    time, strings/s, whole-sort algorithmic bytes against the HBM peak, and the
    dominant kernel with its own roofline."""
    import workloads as W
    out = {}
    cases = [
        ("no_lcp_64Mi", lambda: W.no_lcp(n=64 * 1024 * 1024, seed=5),
         "n=67,108,864 strings of 16 bytes U[1,255], NUL-terminated, seed 5"),
        ("dna_windows_20M", lambda: W.dna_windows(n=20_000_000, text_len=400_000_000, window=100, seed=3),
         "400,000,000-byte text U{A,C,G,T}, n=20,000,000 windows of 100 bytes, seed 3"),
    ]
    for name, gen, desc in cases:
        ss = gen()
        n = ss.n
        chars = torch.from_numpy(ss.chars).to(dev)
        offsets = torch.from_numpy(ss.offsets.view(np.int64)).to(dev)
        perm = torch.empty(n, dtype=torch.int32, device=dev)
        lcp = torch.empty(n, dtype=torch.int32, device=dev)

        def run():
            if ss.fixed_len:
                P.ss_sort_ex(chars, offsets, None, ss.fixed_len, n, perm, lcp, stream=stream)
            else:
                P.ss_sort(chars, offsets, n, perm, lcp, stream=stream)

        for _ in range(2):
            run()
        torch.cuda.synchronize(dev)
        reps = 5
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            run()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        P.profile_reset()
        P.profile_enable(True)
        run()
        torch.cuda.synchronize(dev)
        P.profile_enable(False)
        prof = P.profile_read()
        D, balg = d_and_balg(lcp.cpu().numpy().view(np.uint32))
        dom = max((k for k in prof if BYTES_PER_UNIT.get(k)), key=lambda k: prof[k][1])
        nl, tms, units = prof[dom]
        bpu = BYTES_PER_UNIT.get(dom)
        ach = units * bpu / (tms / 1e3) / 1e9 if bpu else None
        kinds = {"no_lcp_64Mi": "no_lcp", "dna_windows_20M": "dna_windows"}
        kern = {k: {"launches": v[0], "ms": v[1], "units": v[2]} for k, v in prof.items()}
        radix = library_radix_context(P, torch, dev, stream, chars, offsets, n) if name == "no_lcp_64Mi" else None
        compressed = (alphabet_compressed(P, torch, dev, stream, chars, offsets, ss, perm, lcp)
                      if name == "dna_windows_20M" else None)
        cls_cmp = compare_classifiers(P, torch, dev, stream, [dict(chars=chars, offsets=offsets, lengths=None,
                                                                   fixed_len=ss.fixed_len, n=n, perm_out=perm,
                                                                   lcp_out=lcp)])
        out[name] = {"workload": desc, "n": n, "ms": ms, "strings_per_s": n / (ms / 1e3),
                     "d_gb_per_s": D / (ms / 1e3) / 1e9,
                     "whole_sort_roofline": {"algorithmic_bytes": balg, "achieved_gbs": balg / (ms / 1e3) / 1e9,
                                             "frac": balg / (ms / 1e3) / 1e9 / peak},
                     "dominant_kernel": {"kernel": dom, "ms": tms, "share": tms / sum(v[1] for v in prof.values()),
                                         "launches": nl, "units_per_launch": units / max(nl, 1),
                                         "bytes_per_unit": bpu, "achieved_gbs": ach,
                                         "frac": (ach / peak) if ach else None,
                                         "traffic": dram_traffic(dom, kinds[name], units / max(nl, 1))},
                     "kernels": kern,
                     "classifiers": cls_cmp}
        if radix:
            out[name]["library_radix_sort_context"] = radix
        if compressed:
            out[name]["alphabet_compressed"] = compressed
        del chars, offsets, perm, lcp
        torch.cuda.empty_cache()
    return out


def alphabet_compressed(P, torch, dev, stream, chars, offsets, ss, perm, lcp, reps=5):
    """The same DNA windows sorted with alphabet compression (keys of 32
    two-bit characters, Section 8.1): median time, and whether the arrays
    equal the byte-key sort's (which perm / lcp hold on entry)."""
    ref = torch.cat([perm, lcp]).clone()
    q = [dict(chars=chars, offsets=offsets, lengths=None, fixed_len=ss.fixed_len, n=ss.n, perm_out=perm, lcp_out=lcp)]
    tun = [(0, 0, 0, P.alphabet(b"ACGT"))]
    for _ in range(2):
        P.ss_sort_batch_tuned(q, tun, stream=stream)
    torch.cuda.synchronize(dev)
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.ss_sort_batch_tuned(q, tun, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ts.append(e0.elapsed_time(e1))
    ms = float(np.median(ts))
    return {"ms": ms, "strings_per_s": ss.n / (ms / 1e3), "alphabet": "ACGT, 2 bits per character",
            "outputs_equal_byte_keys": bool(torch.equal(torch.cat([perm, lcp]), ref))}


def library_radix_context(P, torch, dev, stream, chars, offsets, n, reps=5):
    """Context only: a library radix sort (torch.sort, stable, on CUDA) of
    each string's first 8 bytes as a 64-bit key with the string indices, the
    keys gathered by ss_gather_keys.  It orders by 8 characters only and
    returns no LCPs, so it is not a string sort; it shows what one pass of a
    tuned 64-bit key sort costs on the same device."""
    depth = torch.zeros(n, dtype=torch.int32, device=dev)
    keys = torch.empty(n, dtype=torch.int64, device=dev)
    P.ss_gather_keys(chars, offsets, None, 0, n, depth, keys, stream=stream)
    skeys = keys ^ torch.tensor(-(1 << 63), dtype=torch.int64, device=dev)   # unsigned order as signed
    with torch.cuda.stream(stream):
        for _ in range(2):
            torch.sort(skeys, stable=True)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            torch.sort(skeys, stable=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    del depth, keys, skeys
    return {"ms": ms, "keys_per_s": n / (ms / 1e3),
            "what": "torch.sort(stable) of the 64-bit first-8-byte keys with indices: a library radix sort, "
                    "8 characters only, no LCPs; context, not a target"}


def compare_merge_methods(P, torch, dev, stream, chars, offsets, rperm, rlcp, rb, perm, lcp, reps=5, fixed_len=0,
                          cache=None):
    """The step's merge with each method of ss_merge_ex (pairwise rounds, the
    default; one pass with LCP loser trees) and, given the runs' sort caches,
    ss_merge_cached (the step's merge): median time of the call, the kernels'
    times from the library's launch events, and whether the outputs equal the
    default's (which perm / lcp hold on entry)."""
    ref = torch.cat([perm, lcp]).clone()
    out = {}
    methods = [(P.MERGE_PAIRWISE, "pairwise_rounds"), (P.MERGE_LOSER_TREE, "loser_tree")]
    if cache is not None:
        methods.append((None, "pairwise_from_sort_caches"))
    for method, name in methods:
        def m():
            if method is None:
                P.ss_merge_cached(chars, offsets, None, fixed_len, rperm, rlcp, *cache, rb, perm, lcp,
                                  run_base=rb[:-1], stream=stream)
                return
            P.ss_merge_ex(chars, offsets, None, fixed_len, rperm, rlcp, rb, perm, lcp, run_base=rb[:-1], method=method,
                          stream=stream)
        m()
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            m()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1))
        P.profile_reset()
        P.profile_enable(True)
        m()
        torch.cuda.synchronize(dev)
        P.profile_enable(False)
        prof = P.profile_read()
        out[name] = {"ms": float(np.median(ts)), "kernels_ms": {k: round(v[1], 4) for k, v in prof.items()},
                     "outputs_equal_default": bool(torch.equal(torch.cat([perm, lcp]), ref))}
    perm.copy_(ref[:perm.shape[0]])
    lcp.copy_(ref[perm.shape[0]:])
    return out


CLASSIFIERS = ("unroll", "equal", "jump")


def compare_classifiers(P, torch, dev, stream, reqs, reps=5):
    """The same requests sorted with each classifier (one ss_sort_batch_tuned
    call): median time of the call, the classification kernels' time per call
    from the library's launch events, and whether the outputs equal the
    default classifier's."""
    out, ref = {}, None
    for cls, name in enumerate(CLASSIFIERS):
        tun = [(0, 0, cls)] * len(reqs)
        P.ss_sort_batch_tuned(reqs, tun, stream=stream)
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            P.ss_sort_batch_tuned(reqs, tun, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1))
        P.profile_reset()
        P.profile_enable(True)
        P.ss_sort_batch_tuned(reqs, tun, stream=stream)
        torch.cuda.synchronize(dev)
        P.profile_enable(False)
        prof = P.profile_read()
        res = torch.cat([torch.cat([q["perm_out"], q["lcp_out"]]) for q in reqs]).clone()
        if ref is None:
            ref = res
        out[name] = {"sort_ms": float(np.median(ts)),
                     "classify_ms": prof.get("classify", (0, 0.0, 0))[1],
                     "jump_tables_ms": prof.get("jump_tables", (0, 0.0, 0))[1],
                     "classify_launches": prof.get("classify", (0, 0.0, 0))[0],
                     "outputs_equal_unroll": bool(torch.equal(res, ref))}
    return out


def batched_vs_plain(P, torch, dev, stream, nreq=4096, seed=4):
    """The batched configuration: nreq independent requests of log-uniform sizes
    1,000..1,000,000 strings, generators random / URL-like / DNA-like by request
    number mod 3, all arriving at once.  Batched = one ss_sort_batch call for all
    of them; plain = one ss_sort call per request, in arrival order.  Latency of a
    request = its completion time from the common arrival (the batch completes
    every request at its end).  Each request is a contiguous slice of a seeded
    pool of its generator (own offsets, shared bytes)."""
    import workloads as W
    rng = np.random.default_rng(seed)
    pools = [W.random_lower(2_000_000, seed=seed * 10 + 0), W.url_like(2_000_000, seed=seed * 10 + 1),
             W.dna_windows(2_000_000, 40_000_000, 100, seed=seed * 10 + 2)]
    dpools = [(torch.from_numpy(p.chars).to(dev), torch.from_numpy(p.offsets.view(np.int64)).to(dev), p) for p in pools]
    sizes = np.floor(np.exp(rng.uniform(np.log(1e3), np.log(1e6), nreq))).astype(np.int64)
    starts = [int(rng.integers(0, pools[r % 3].n - int(sizes[r]) + 1)) for r in range(nreq)]
    total = int(sizes.sum())
    base = np.concatenate([[0], np.cumsum(sizes)])
    perm_b = torch.empty(total, dtype=torch.int32, device=dev)
    lcp_b = torch.empty(total, dtype=torch.int32, device=dev)
    perm_p = torch.empty(total, dtype=torch.int32, device=dev)
    lcp_p = torch.empty(total, dtype=torch.int32, device=dev)

    def req(r, perm, lcp):
        chars, offs, pool = dpools[r % 3]
        n = int(sizes[r])
        return dict(chars=chars, offsets=offs[starts[r]:starts[r] + n], lengths=None, fixed_len=pool.fixed_len, n=n,
                    perm_out=perm[int(base[r]):int(base[r + 1])], lcp_out=lcp[int(base[r]):int(base[r + 1])])

    breqs = [req(r, perm_b, lcp_b) for r in range(nreq)]
    preqs = [req(r, perm_p, lcp_p) for r in range(nreq)]
    # one tuning per generator, picked by the library's autotuner on a 1 M sample of its pool
    tuned = []
    for g in range(3):
        chars, offs, pool = dpools[g]
        q = dict(chars=chars, offsets=offs, lengths=None, fixed_len=pool.fixed_len, n=pool.n, perm_out=perm_b,
                 lcp_out=lcp_b)
        tuned.append(P.ss_autotune(q, sample_n=1_000_000, stream=stream)[0])
    tunings = [tuned[r % 3] for r in range(nreq)]
    P.ss_sort_batch(breqs, stream=stream)   # warm-up (pool growth, attributes)
    torch.cuda.synchronize(dev)
    bt = []
    for _ in range(2):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.ss_sort_batch(breqs, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        bt.append(e0.elapsed_time(e1))
    P.ss_sort_batch_tuned(breqs, tunings, stream=stream)
    torch.cuda.synchronize(dev)
    tt = []
    for _ in range(2):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.ss_sort_batch_tuned(breqs, tunings, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        tt.append(e0.elapsed_time(e1))
    tuned_perm, tuned_lcp = perm_b.clone(), lcp_b.clone()
    P.ss_sort_batch(breqs, stream=stream)   # the default-tuned result stays in perm_b / lcp_b
    torch.cuda.synchronize(dev)
    tuned_same = bool(torch.equal(tuned_perm, perm_b) and torch.equal(tuned_lcp, lcp_b))
    del tuned_perm, tuned_lcp
    for r in range(0, nreq, 97):   # warm-up of the one-request path
        q = preqs[r]
        if q["fixed_len"]:
            P.ss_sort_ex(q["chars"], q["offsets"], None, q["fixed_len"], q["n"], q["perm_out"], q["lcp_out"], stream=stream)
        else:
            P.ss_sort(q["chars"], q["offsets"], q["n"], q["perm_out"], q["lcp_out"], stream=stream)
    torch.cuda.synchronize(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(nreq + 1)]
    ev[0].record(stream)
    for r in range(nreq):
        q = preqs[r]
        if q["fixed_len"]:
            P.ss_sort_ex(q["chars"], q["offsets"], None, q["fixed_len"], q["n"], q["perm_out"], q["lcp_out"], stream=stream)
        else:
            P.ss_sort(q["chars"], q["offsets"], q["n"], q["perm_out"], q["lcp_out"], stream=stream)
        ev[r + 1].record(stream)
    torch.cuda.synchronize(dev)
    done = np.array([ev[0].elapsed_time(ev[r + 1]) for r in range(nreq)])
    service = np.diff(np.concatenate([[0.0], done]))
    equal = bool(torch.equal(perm_b, perm_p) and torch.equal(lcp_b, lcp_p))
    tb = float(np.median(bt))
    tp = float(done[-1])
    out = {
        "workload": f"{nreq} requests, sizes log-uniform 1,000..1,000,000 strings, generators random/URL-like/DNA-like by request mod 3, seed {seed}; all arrive at once",
        "requests": nreq, "strings": total,
        "batched": {"ms": tb, "strings_per_s": total / (tb / 1e3), "latency_p50_ms": tb, "latency_p99_ms": tb,
                    "launches": "one ss_sort_batch call"},
        "plain": {"ms": tp, "strings_per_s": total / (tp / 1e3),
                  "latency_p50_ms": float(np.percentile(done, 50)), "latency_p99_ms": float(np.percentile(done, 99)),
                  "service_p50_ms": float(np.percentile(service, 50)), "service_p99_ms": float(np.percentile(service, 99)),
                  "launches": "one ss_sort per request, in arrival order"},
        "speedup": tp / tb,
        "autotuned": {"tunings_by_generator": {n_: {"child_target": t[0], "min_step": t[1],
                                                    "classifier": ["unroll", "equal", "jump"][t[2]],
                                                    "alphabet": t[3], "max_depth": t[4], "small_max": t[5]}
                                                for n_, t in zip(["random", "url_like", "dna_like"], tuned)},
                      "ms": float(np.median(tt)), "strings_per_s": total / (float(np.median(tt)) / 1e3),
                      "how": "ss_autotune on a 1 M sample of each generator's pool, then one ss_sort_batch_tuned call",
                      "outputs_equal_default": tuned_same},
        "outputs_equal": equal,
    }
    del perm_b, lcp_b, perm_p, lcp_p, dpools
    torch.cuda.empty_cache()
    return out


def _output_hash(torch, perm, lcp, chunk=1 << 28):
    """Two 64-bit sums over positions i of the outputs (wrapping int64
    arithmetic), taken in chunks: equal hashes of two runs stand for equal
    outputs without holding both on the device."""
    h1 = torch.zeros((), dtype=torch.int64, device=perm.device)
    h2 = torch.zeros((), dtype=torch.int64, device=perm.device)
    n = perm.shape[0]
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        i = torch.arange(a, b, dtype=torch.int64, device=perm.device)
        p_ = perm[a:b].to(torch.int64) & 0xFFFFFFFF
        l_ = lcp[a:b].to(torch.int64) & 0xFFFFFFFF
        h1 += ((p_ + 1) * (i * 2 + 1) * 0x9E3779B1 + (l_ + 7) * 0x85EBCA77).sum()
        h2 += ((p_ * 0xC2B2AE3D + 3) * (l_ * 2 + 1) + i * 0x27D4EB2F).sum()
        del i, p_, l_
    return (int(h1.item()), int(h2.item()))


def serving_vs_plain(P, torch, dev, url_chars, url_offsets, capacity_sps, nreq=20000, loads=(0.7, 0.5, 0.9, 1.1),
                     seed=5, workers=3):
    """The serving configuration: requests of log-uniform sizes 1,000..4,000,000
    strings (generators random / URL-like / DNA-like by request mod 3) arrive as
    a Poisson stream whose offered load is a multiple of the batched capacity
    measured before (strings/s), plus one no-LCP job of 64 Mi strings in the
    middle.  Served = the continuous-batching server (`workers` streams, 120 GB
    budget), at the first load and at each of the others; plain = the first
    load's stream through a server with one worker and batches of one request
    (one request per launch sequence).  Latency = completion - arrival, on the
    server's clock.  Every run writes the same output arrays; their hashes
    are compared run against run (outputs_equal)."""
    import threading
    import workloads as W
    rng = np.random.default_rng(seed)
    lower = W.random_lower(4_000_000, seed=seed * 10)
    dna = W.dna_windows(4_000_000, 80_000_000, 100, seed=seed * 10 + 2)
    nolcp = W.no_lcp(n=64 * 1024 * 1024, seed=5)
    pools = [(torch.from_numpy(lower.chars).to(dev), torch.from_numpy(lower.offsets.view(np.int64)).to(dev), 0,
              lower.n),
             (url_chars, url_offsets, 0, int(url_offsets.shape[0])),
             (torch.from_numpy(dna.chars).to(dev), torch.from_numpy(dna.offsets.view(np.int64)).to(dev), 100, dna.n)]
    big = (torch.from_numpy(nolcp.chars).to(dev), torch.from_numpy(nolcp.offsets.view(np.int64)).to(dev), 0, nolcp.n)
    sizes = np.floor(np.exp(rng.uniform(np.log(1e3), np.log(4e6), nreq))).astype(np.int64)
    src = [pools[r % 3] for r in range(nreq)]
    starts = [int(rng.integers(0, src[r][3] - int(sizes[r]) + 1)) for r in range(nreq)]
    mid = nreq // 2
    sizes = np.insert(sizes, mid, big[3])
    src.insert(mid, big)
    starts.insert(mid, 0)
    nall = len(sizes)
    total = int(sizes.sum())
    unit_gaps = rng.exponential(1.0, nall)   # one arrival pattern, scaled per offered load
    base = np.concatenate([[0], np.cumsum(sizes)])
    perm = torch.empty(total, dtype=torch.int32, device=dev)
    lcp = torch.empty(total, dtype=torch.int32, device=dev)
    reqs = []
    for r in range(nall):
        chars, offs, fixed, _ = src[r]
        n = int(sizes[r])
        reqs.append(dict(chars=chars, offsets=offs[starts[r]:starts[r] + n], lengths=None, fixed_len=fixed, n=n,
                         perm_out=perm[int(base[r]):int(base[r + 1])], lcp_out=lcp[int(base[r]):int(base[r + 1])]))

    def run(workers_, max_batch, load):
        rate = load * capacity_sps / float(sizes.mean())   # requests per second
        gaps = unit_gaps / rate
        perm.fill_(-1)
        lcp.fill_(-1)
        torch.cuda.synchronize(dev)
        tickets = [None] * nall
        with P.Server(120 << 30, workers=workers_, max_batch=max_batch) as srv:
            def producer():
                t_next = time.perf_counter()
                for r in range(nall):
                    t_next += float(gaps[r])
                    d = t_next - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                    tickets[r] = srv.submit(reqs[r])
            th = threading.Thread(target=producer)
            th.start()
            th.join()
            res = [srv.wait(t) for t in tickets]
        st = [s_ for s_, _ in res]
        tm = np.array([t_ for _, t_ in res])
        lat = tm[:, 2] - tm[:, 0]
        span = float(tm[:, 2].max() - tm[:, 0].min())
        torch.cuda.synchronize(dev)
        out = {"offered_load": load, "arrival_rate_per_s": rate, "makespan_ms": span,
               "strings_per_s": total / (span / 1e3),
               "latency_p50_ms": float(np.percentile(lat, 50)), "latency_p99_ms": float(np.percentile(lat, 99)),
               "latency_64Mi_job_ms": float(lat[mid]), "errors": int(sum(1 for x in st if x != 0)),
               "batches": int(len(set(tm[:, 1].tolist())))}
        return out, _output_hash(torch, perm, lcp)

    served, h_served = run(workers, 0, loads[0])
    plain, h_plain = run(1, 1, loads[0])
    sweep, sweep_equal = [], True
    for ld in loads[1:]:
        o, h = run(workers, 0, ld)
        sweep.append(o)
        sweep_equal = sweep_equal and h == h_served
    del perm, lcp, reqs, pools, big
    torch.cuda.empty_cache()
    return {
        "workload": (f"{nreq} requests, sizes log-uniform 1,000..4,000,000 strings, generators random/URL-like/DNA-like "
                     f"by request mod 3, Poisson arrivals at {loads[0]:.1f} x the batched capacity, plus one no-LCP "
                     f"job of 64 Mi strings in the middle; seed {seed}"),
        "requests": nall, "strings": total, "budget_bytes": 120 << 30,
        "served": dict(served, workers=workers, batching="continuous: every idle worker takes all admitted waiting requests"),
        "plain": dict(plain, workers=1, batching="one request per launch sequence, first come first served"),
        "load_sweep": sweep,
        "outputs_equal": bool(h_served == h_plain and sweep_equal),
        "outputs_compared": "two 64-bit position-weighted sums of every run's perm and lcp arrays",
    }


def aggregate(dist, ms, units, device):
    """Replicas (one process per GPU, no collective on the data path): the job's
    time is the slowest rank's, its work the sum of all ranks' units."""
    if dist is None:
        return ms, units
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(u.item()))


def dram_traffic(kernel, workload_kind, units_per_launch):
    """DRAM bytes (read + write) per launch of `kernel`: the bytes per unit
    that one small-case ncu capture of that kernel measured (profiles/traffic.json),
    times the units of a full launch.  None when the sources changed since the
    capture, or the capture was taken on another kind of workload."""
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(tp) as f:
            tj = json.load(f)
    except Exception:
        return None
    if tj.get("source_hash") != _source_hash():
        return None
    k = tj.get("kernels", {}).get(workload_kind, {}).get(kernel)
    if not k or k.get("workload_kind") != workload_kind:
        return None
    return float(k["dram_bytes_per_unit"]) * float(units_per_launch)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


WORKLOADS = {   # name: default n (the configuration's size)
    "url_like": 10_000_000,
    "no_lcp": 64 * 1024 * 1024,
    "dna_windows": 20_000_000,
}


def workload(n, kind="url_like"):
    import workloads as W
    if kind == "no_lcp":
        return W.no_lcp(n=n, seed=5)
    if kind == "dna_windows":
        return W.dna_windows(n=n, text_len=20 * n, window=100, seed=3)
    return W.url_like(n, seed=2)


def workload_name(n, runs, kind="url_like"):
    what = {
        "url_like": (f"url_like: n={n:,} strings 'http://' + host (2,000 hosts, Zipf s=1.1) + 1-6 path segments, "
                     f"5% duplicates, seed 2"),
        "no_lcp": f"no_lcp: n={n:,} strings of 16 bytes U[1,255], NUL-terminated, seed 5",
        "dna_windows": f"dna_windows: text of {20 * n:,} bytes U{{A,C,G,T}}, n={n:,} windows of 100 bytes, seed 3",
    }[kind]
    return f"{what}; sorted as {runs} runs + {runs}-way LCP merge"


def d_and_balg(lcp: np.ndarray):
    """D (Section 2) and the algorithmic bytes of a whole sort from the output LCP array."""
    l = lcp.astype(np.int64)
    nxt = np.concatenate([l[1:], [0]])
    prv = l.copy()
    prv[0] = 0
    dist = np.maximum(prv, nxt) + 1
    D = int(dist.sum())
    n = l.shape[0]
    balg = 8 * n + int((8 * ((dist + 7) // 8)).sum()) + 8 * n
    return D, balg


class Clocks:
    """nvidia-smi samples (every 20 ms, time-stamped) around the timed region;
    the summary keeps the samples that fall inside it (the nearest one if the
    region is shorter than the sampling interval)."""

    def __init__(self, index):
        self.proc = None
        # raw samples go to $SS_BENCH_OUT (default: bench_out/ in the repository)
        out = os.environ.get("SS_BENCH_OUT", os.path.join(ROOT, "bench_out"))
        self.path = os.path.join(out, f"clocks_rank{index}.csv")
        self.index = index
        self.t0 = self.t1 = None

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.f, stderr=subprocess.DEVNULL)
            deadline = time.time() + 10.0   # wait for the first sample: the sampler is up
            while time.time() < deadline and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def mark(self, begin):
        if begin:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        import datetime
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[1]), float(parts[2]),
                             {nm for k, nm in enumerate(names) if parts[5 + k].lower() == "active"}))
            except ValueError:
                continue
        if not rows:
            return None
        inside = [r for r in rows if self.t0 is not None and self.t0 <= r[0] <= (self.t1 or r[0])]
        if not inside and self.t0 is not None:
            mid = 0.5 * (self.t0 + (self.t1 or self.t0))
            inside = [min(rows, key=lambda r: abs(r[0] - mid))]
        sm = [r[1] for r in inside]
        reasons = set().union(*[r[3] for r in inside]) if inside else set()
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(r[2] for r in inside), "reasons": sorted(reasons),
                "samples": len(inside), "interval_ms": 20}


def cpu_baseline(ss, seconds):
    """The oracle (one thread) on the first m strings of the workload, m sized for ~`seconds`."""
    import oracle
    import workloads as W
    m = min(ss.n, 200_000)
    t0 = time.perf_counter()
    oracle.sort(W.subset(ss, np.arange(m)))
    dt = time.perf_counter() - t0
    if m < ss.n and dt < seconds:
        m2 = min(ss.n, int(m * seconds / max(dt, 1e-3) / 1.1))
        if m2 > m:
            m = m2
            t0 = time.perf_counter()
            oracle.sort(W.subset(ss, np.arange(m)))
            dt = time.perf_counter() - t0
    return {"value": m / dt, "unit": "strings/s", "cores": 1, "kind": "oracle",
            "sample": f"first {m:,} strings of the workload, one qsort + naive LCP pass ({dt:.1f} s)"}


def cpu_parallel(ss):
    """Context beside the oracle: the same order from a parallel library
    stable sort (libstdc++ parallel mode, OpenMP) on all host cores, on the
    whole workload."""
    import oracle
    try:
        t0 = time.perf_counter()
        _, _, used = oracle.sort_parallel(ss, threads=os.cpu_count() or 1)
        dt = time.perf_counter() - t0
    except Exception as e:   # no g++/OpenMP on this host
        return {"unavailable": f"parallel CPU baseline not built: {e}"}
    return {"value": ss.n / dt, "unit": "strings/s", "cores": used,
            "kind": "library parallel stable sort with the oracle's comparator + naive LCP",
            "sample": f"the whole workload, {ss.n:,} strings ({dt:.1f} s)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    import workloads as W
    oracle.build()
    ss = workload(args.n, args.workload)
    m = min(ss.n, 1_000_000)
    sub = W.subset(ss, np.arange(m))
    for _ in range(max(0, args.warmup)):
        oracle.sort(W.subset(ss, np.arange(min(m, 100_000))))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sort(sub)
    dt = time.perf_counter() - t0
    value = m * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "strings/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": workload_name(args.n, args.runs, args.workload), "sample": m},
            "cpu_baseline": {"value": value, "unit": "strings/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {m:,} strings of the workload per step"},
            "e2e": {"value": value, "unit": "strings/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.n <= 0:
        args.n = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1403_2056_gb300 as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    ss = workload(args.n, args.workload)
    n, K = ss.n, args.runs
    chars = torch.from_numpy(ss.chars).to(dev)
    offsets = torch.from_numpy(ss.offsets.view(np.int64)).to(dev)
    rb = np.array([n * k // K for k in range(K + 1)], np.uint32)
    rperm = torch.empty(n, dtype=torch.int32, device=dev)
    rlcp = torch.empty(n, dtype=torch.int32, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    lcp = torch.empty(n, dtype=torch.int32, device=dev)
    roff = torch.empty(n, dtype=torch.int64, device=dev)   # the runs' caches, from their sort to the merge
    rck = torch.empty(n, dtype=torch.int64, device=dev)
    rckd = torch.empty(n, dtype=torch.int32, device=dev)
    fl = ss.fixed_len
    reqs = [dict(chars=chars, offsets=offsets[int(rb[k]):int(rb[k + 1])], lengths=None, fixed_len=fl,
                 n=int(rb[k + 1] - rb[k]), perm_out=rperm[int(rb[k]):int(rb[k + 1])],
                 lcp_out=rlcp[int(rb[k]):int(rb[k + 1])]) for k in range(K)]
    caches = [(roff[int(rb[k]):int(rb[k + 1])], rck[int(rb[k]):int(rb[k + 1])], rckd[int(rb[k]):int(rb[k + 1])])
              for k in range(K)]
    stream = torch.cuda.current_stream(dev)

    def step():
        P.ss_sort_batch_cached(reqs, caches, stream=stream)
        P.ss_merge_cached(chars, offsets, None, fl, rperm, rlcp, roff, rck, rckd, rb, perm, lcp, run_base=rb[:-1],
                          stream=stream)

    def sort_only():
        P.ss_sort_ex(chars, offsets, None, fl, n, perm, lcp, stream=stream)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)

    # sort only (rows a1-a9, one request) for context, before the timed region
    ms_sort, calls_ms = None, []
    if not args.capture:
        for _ in range(2):
            sort_only()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = max(3, args.steps // 2)
        e0.record(stream)
        for _ in range(reps):
            t0 = time.perf_counter()
            sort_only()
            calls_ms.append((time.perf_counter() - t0) * 1e3)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_sort = e0.elapsed_time(e1) / reps
        for _ in range(2):
            step()
        torch.cuda.synchronize(dev)

    # timed region: exactly K steps between a barrier and a synchronize on both
    # sides, CUDA events on the launch stream, clocks sampled
    clocks = Clocks(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize(dev)
    launches0 = P.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks.mark(True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clocks.mark(False)
    barrier()
    launches = P.launch_count() - launches0
    ck = clocks.stop()
    ms, job_strings = aggregate(dist, ev0.elapsed_time(ev1) / args.steps, n, dev)

    # per-kernel times: the same K steps again with the library's launch events on
    # (the base-case size classes then run one after another, so every kernel's
    # time is its own)
    P.profile_reset()
    P.profile_enable(True)
    pe0 = torch.cuda.Event(enable_timing=True)
    pe1 = torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    for _ in range(args.steps):
        step()
    pe1.record(stream)
    torch.cuda.synchronize(dev)
    P.profile_enable(False)
    prof = P.profile_read()
    profiled_ms = pe0.elapsed_time(pe1) / args.steps

    lcp_h = lcp.cpu().numpy().view(np.uint32)
    D, balg = d_and_balg(lcp_h)
    value = job_strings / (ms / 1e3)

    # dominant kernel and its roofline
    peak, peak_kind = load_peaks()
    kernels = {}
    for name, (nl, tms, units) in prof.items():
        bpu = BYTES_PER_UNIT.get(name)
        gbs = (units * bpu / (tms / 1e3) / 1e9) if (bpu and tms > 0) else None
        kernels[name] = {"launches": nl, "ms_per_step": tms / args.steps, "share": None,
                         "units_per_launch": units / max(nl, 1), "bytes_per_unit": bpu,
                         "achieved_gbs": gbs}
    tot = sum(v["ms_per_step"] for v in kernels.values()) or 1.0
    for v in kernels.values():
        v["share"] = v["ms_per_step"] / tot
    # the dominant kernel among those that move a step's data (a kernel that
    # only searches, such as the merge's chunk starts, has no algorithmic bytes);
    # the overall top kernel is named beside it
    top = max(kernels, key=lambda k: kernels[k]["ms_per_step"]) if kernels else None
    moving = [k for k in kernels if kernels[k]["bytes_per_unit"]]
    dom = max(moving, key=lambda k: kernels[k]["ms_per_step"]) if moving else None
    roofline = None
    if dom:
        kd = kernels[dom]
        ach = kd["achieved_gbs"] or 0.0
        roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak, "peak_kind": peak_kind,
                    "traffic": dram_traffic(dom, args.workload, kd["units_per_launch"]),
                    "units_per_launch": kd["units_per_launch"], "bytes_per_unit": kd["bytes_per_unit"],
                    "algorithmic_bytes_per_launch": kd["units_per_launch"] * (kd["bytes_per_unit"] or 0),
                    "launch_ms": kd["ms_per_step"] * args.steps / max(kd["launches"], 1),
                    "carried_bytes_per_unit": CARRIED_BYTES_PER_UNIT.get(dom, 0),
                    "top_kernel": {"kernel": top, "share": kernels[top]["share"],
                                   "bytes_per_unit": kernels[top]["bytes_per_unit"]},
                    "whole_step": {"algorithmic_bytes": balg, "frac": balg / (ms / 1e3) / 1e9 / peak}}

    line = {
        "metric": METRIC, "value": value, "unit": "strings/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": workload_name(n, K, args.workload), "n": n, "N_bytes": int(ss.chars.nbytes),
                   "mean_len": ss.meta.get("mean_len"), "runs": K, "parallelism": f"replicas x{world}",
                   "l2": (f"inputs larger than L2 (chars {ss.chars.nbytes / 1e9:.2f} GB + offsets "
                          f"{ss.offsets.nbytes / 1e6:.0f} MB per step)"
                          if ss.chars.nbytes + ss.offsets.nbytes > L2_BYTES else
                          "inputs smaller than L2: not a valid bench configuration")},
        "d_gb_per_s": D * (job_strings // n) / (ms / 1e3) / 1e9, "D": D,
        "whole_sort_roofline": {"algorithmic_bytes": balg, "achieved_gbs": balg / (ms / 1e3) / 1e9,
                                "frac": balg / (ms / 1e3) / 1e9 / peak},
        "sort_only": {"ms": ms_sort, "value": (n / (ms_sort / 1e3)) if ms_sort else None, "unit": "strings/s",
                      "calls_ms": [round(x, 3) for x in calls_ms],
                      "what": "one ss_sort of the whole set (no runs, no merge)"},
        "roofline": roofline,
        "gpu_launches": int(launches),
        "clocks": ck,
        "kernels": kernels,
        "kernels_pass": {"ms_per_step": profiled_ms,
                         "what": "the per-kernel table and the roofline come from a second pass of the same K steps "
                                 "with launch events on and the base-case classes serialised"},
    }

    # end to end through the host-buffer API: H2D, sort runs + merge, D2H
    if not args.no_e2e:
        hc = torch.from_numpy(ss.chars).pin_memory()
        ho = torch.from_numpy(ss.offsets.view(np.int64)).pin_memory()
        hp = torch.empty(n, dtype=torch.int32).pin_memory()
        hl = torch.empty(n, dtype=torch.int32).pin_memory()
        for _ in range(2):
            P.ss_sort_host(hc, ho, None, fl, hp, hl, runs=K, stream=stream)
        barrier()
        torch.cuda.synchronize(dev)
        # each call returns when its outputs are on the host: the median of the
        # calls' wall times (a few calls now and then take longer on the host)
        reps = max(10, args.steps)
        call_ms = []
        for _ in range(reps):
            t0 = time.perf_counter()
            P.ss_sort_host(hc, ho, None, fl, hp, hl, runs=K, stream=stream)
            call_ms.append((time.perf_counter() - t0) * 1e3)
        torch.cuda.synchronize(dev)
        one_ms, _ = aggregate(dist, float(np.median(call_ms)), n, dev)
        same = np.array_equal(hp.numpy(), perm.cpu().numpy()) and np.array_equal(hl.numpy(), lcp.cpu().numpy())
        # the same steps as a stream of host requests through the server: each
        # step still copies its inputs in and its result out, and one step's
        # copies overlap another step's sort
        outs = [(torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty(n, dtype=torch.int32).pin_memory())
                for _ in range(max(1, args.e2e_inflight))]
        with P.Server(64 << 30, workers=args.e2e_workers) as srv:
            for k in range(2):
                o = outs[k % len(outs)]
                srv.wait(srv.submit_host(hc, ho, None, fl, o[0], o[1], runs=K))
            barrier()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            inflight = []
            reps_p = args.e2e_steps if args.e2e_steps > 0 else max(30, args.steps)
            for i in range(reps_p):
                if len(inflight) == len(outs):
                    st_, _ = srv.wait(inflight.pop(0))
                    same = same and st_ == 0
                o = outs[i % len(outs)]
                inflight.append(srv.submit_host(hc, ho, None, fl, o[0], o[1], runs=K))
            for t_ in inflight:
                st_, _ = srv.wait(t_)
                same = same and st_ == 0
            pipe_ms, e2e_strings = aggregate(dist, (time.perf_counter() - t0) / reps_p * 1e3, n, dev)
        same = same and all(np.array_equal(o[0].numpy(), hp.numpy()) and np.array_equal(o[1].numpy(), hl.numpy())
                            for o in outs)
        line["e2e"] = {"value": e2e_strings / (pipe_ms / 1e3), "unit": "strings/s",
                       "h2d_bytes_per_step": int(ss.chars.nbytes + 8 * n), "d2h_bytes_per_step": int(8 * n),
                       "ms_per_step": pipe_ms, "steps": reps_p,
                       "api": (f"ss_server_submit_host ({args.e2e_workers} workers, up to {len(outs)} steps in "
                               f"flight): copies in, sort of {K} runs + merge, copies out per step"),
                       "single_call": {"api": "ss_sort_host, one call per step", "ms_per_step": one_ms,
                                       "value": e2e_strings / (one_ms / 1e3), "calls": reps,
                                       "what": "median of the calls' wall times; max " + f"{max(call_ms):.2f} ms"},
                       "equals_device_result": bool(same)}

    if rank == 0 and not args.no_extra:
        line["merge_methods"] = dict(what="the step's merge of its runs by each method of ss_merge_ex, and from the "
                                          "runs' sort caches (ss_merge_cached, the step's merge)",
                                     **compare_merge_methods(P, torch, dev, stream, chars, offsets, rperm, rlcp, rb,
                                                             perm, lcp, fixed_len=fl, cache=(roff, rck, rckd)))
        line["classifiers"] = dict(what="the step's 4 runs sorted by one ss_sort_batch_tuned call per classifier",
                                   **compare_classifiers(P, torch, dev, stream, reqs))
        line["other_workloads"] = other_workloads(P, torch, dev, stream, peak)
        # the 64 Mi no-LCP job's fractions travel in the roofline object itself
        nl_ = line["other_workloads"]["no_lcp_64Mi"]
        if line.get("roofline") is not None:
            line["roofline"]["no_lcp_64Mi"] = {
                "ms": nl_["ms"], "strings_per_s": nl_["strings_per_s"],
                "whole_sort": {"algorithmic_bytes": nl_["whole_sort_roofline"]["algorithmic_bytes"],
                               "achieved": nl_["whole_sort_roofline"]["achieved_gbs"],
                               "frac": nl_["whole_sort_roofline"]["frac"]},
                "kernel": nl_["dominant_kernel"]["kernel"], "achieved": nl_["dominant_kernel"]["achieved_gbs"],
                "frac": nl_["dominant_kernel"]["frac"], "traffic": nl_["dominant_kernel"]["traffic"],
                "bytes_per_unit": nl_["dominant_kernel"]["bytes_per_unit"],
                "units_per_launch": nl_["dominant_kernel"]["units_per_launch"]}
    if rank == 0 and not args.no_batched:
        line["batched"] = batched_vs_plain(P, torch, dev, stream, nreq=args.batched_requests)
        if not args.no_serving and args.workload == "url_like":   # the served mix takes the URL set as a pool
            line["serving"] = serving_vs_plain(P, torch, dev, chars, offsets,
                                               capacity_sps=line["batched"]["batched"]["strings_per_s"],
                                               nreq=args.serving_requests)
    if rank == 0 and not args.no_cpu:
        import oracle
        oracle.build()
        line["cpu_baseline"] = cpu_baseline(ss, args.cpu_seconds)
        line["cpu_parallel"] = cpu_parallel(ss)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _strip_comments(src: str) -> str:
    """C/C++ source without // and /* */ comments (string and character
    literals kept), whitespace runs collapsed: what the compiler sees."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def _source_hash():
    """Hash of the CUDA sources without their comments: DRAM counters taken on
    one revision stay valid across comment-only edits."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1403_2056_gb300", "csrc")
    files = [os.path.join(d, f) for f in sorted(os.listdir(d)) if f.endswith((".cu", ".cuh"))]
    files.append(os.path.join(ROOT, "include", "ss.h"))
    for path in files:
        h.update(os.path.basename(path).encode() + b"\0")
        h.update(_strip_comments(open(path, encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    sys.exit(main())
