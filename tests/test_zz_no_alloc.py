"""The allocation-free scan entry point (GPU, C ABI).

``ab_exclusive_scan_u32_static`` serves callers that cannot allocate device
memory: it keeps its look-back state in a static device array instead of a
context's workspace.  Its output must equal the cell-offset table that the
allocating path (``ab_build``) computes, on two calls in a row (the second
call must not see the first call's leftover state).  The file is named to be
collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _scan_static(lib, counts_dev, out_dev, n):
    st = lib.ab_exclusive_scan_u32_static(ctypes.c_void_p(counts_dev.data_ptr()),
                                          ctypes.c_void_p(out_dev.data_ptr()), n,
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


def test_static_scan_matches_build_cell_table(cuda):
    import paper_1704_08907_gb300 as ab
    from paper_1704_08907_gb300 import _abi
    lib = _abi.load()
    ctx = ab.Context(0)
    results = []
    for w in (synth.c2(n=300000), synth.c1()):
        dom = ab.Domain(w.dim, w.periodic, w.radius)
        ab.ab_build(ctx, dom, torch.from_numpy(w.pos).to(cuda))
        _, start = ab.ab_cell_export(ctx)             # allocating path's table
        ref = start.cpu().numpy().view(np.uint32)
        counts = np.zeros(len(ref), dtype=np.uint32)   # n_cells counts + one 0
        counts[:-1] = np.diff(ref.astype(np.int64)).astype(np.uint32)
        counts_dev = torch.from_numpy(counts.view(np.int32)).to(cuda)
        out_dev = torch.full((len(ref),), -7, dtype=torch.int32, device=cuda)
        assert _scan_static(lib, counts_dev, out_dev, len(ref)) == 0
        got = out_dev.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, ref)
        # in place, on the same buffer
        assert _scan_static(lib, counts_dev, counts_dev, len(ref)) == 0
        assert np.array_equal(counts_dev.cpu().numpy().view(np.uint32), ref)
        results.append(len(ref))
    assert results[0] != results[1]
    ab.ab_sync(ctx)
    ctx.close()


def test_static_scan_rejects_oversize(cuda):
    from paper_1704_08907_gb300 import _abi
    lib = _abi.load()
    buf = torch.zeros(16, dtype=torch.int32, device=cuda)
    p = ctypes.c_void_p(buf.data_ptr())
    assert lib.ab_exclusive_scan_u32_static(p, p, (1 << 24) + 1, None) == 1
    assert lib.ab_exclusive_scan_u32_static(p, ctypes.c_void_p(buf.data_ptr() + 4), 8, None) == 2
