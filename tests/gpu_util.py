"""Helpers for GPU tests: move a StringSet to the device and call the C ABI."""
import numpy as np


def to_device(ss):
    import torch
    dev = torch.device("cuda:0")
    chars = torch.from_numpy(ss.chars).to(dev)
    offsets = torch.from_numpy(ss.offsets.view(np.int64)).to(dev)
    lengths = None if ss.lengths is None else torch.from_numpy(ss.lengths.view(np.int32)).to(dev)
    return chars, offsets, lengths


def gpu_sort(ss, chars=None, offsets=None, lengths=None):
    import torch
    import paper_1403_2056_gb300 as P
    if chars is None:
        chars, offsets, lengths = to_device(ss)
    n = ss.n
    perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda:0")
    lcp = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda:0")
    if lengths is None and ss.fixed_len == 0:
        P.ss_sort(chars, offsets, n, perm, lcp)
    else:
        P.ss_sort_ex(chars, offsets, lengths, ss.fixed_len, n, perm, lcp)
    torch.cuda.synchronize()
    return perm[:n].cpu().numpy().view(np.uint32), lcp[:n].cpu().numpy().view(np.uint32)
