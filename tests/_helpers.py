"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch

import oracle


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def host(t):
    return t.detach().cpu().numpy()


def rel_err(y, ref, den):
    """max |y - ref| / max(|ref|, den), the pair-sum error metric."""
    y = np.asarray(y, np.float64)
    ref = np.asarray(ref, np.float64)
    d = np.maximum(np.abs(ref), np.asarray(den, np.float64))
    d = np.where(d > 0, d, 1.0)
    return float(np.max(np.abs(y - ref) / d)) if y.size else 0.0


def rows_of(offsets, idx, rows):
    """Sorted neighbour rows ``rows`` of a (host) CSR."""
    return [np.sort(idx[offsets[r]:offsets[r + 1]]) for r in rows]


def oracle_box(w):
    return oracle.Box(w.dim, w.periodic, w.lo, w.hi, w.radius)


def gpu_csr_rows(off_dev, idx_dev, rows):
    """Gather rows of a device CSR to the host (sorted by j)."""
    off = host(off_dev)
    idx_h = None
    if idx_dev.numel() < 50_000_000:
        idx_h = host(idx_dev)
    out = []
    for r in rows:
        a, b = int(off[r]), int(off[r + 1])
        seg = idx_h[a:b] if idx_h is not None else host(idx_dev[a:b])
        out.append(np.sort(seg))
    return off, out
