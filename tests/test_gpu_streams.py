"""The library under a caller that overlaps transfers with compute: positions
copied in and forces copied out on the caller's own streams, ordered by
events, while the context computes on its stream.  Every step must give the
same bits as the same steps run one after another on one stream (GPU, C ABI).
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ab():
    import paper_1704_08907_gb300 as ab
    return ab


def _steps(n_steps):
    """Positions of n_steps steps: the same points, each step jittered
    differently (seeded), as packed xyz host arrays."""
    w = synth.c2()
    base = np.ascontiguousarray(w.pos[:200_000, :3])
    g = np.random.default_rng(9)
    out = []
    for _ in range(n_steps):
        p = base + g.uniform(-1e-3, 1e-3, base.shape).astype(np.float32)
        out.append(np.ascontiguousarray(np.mod(p, 1.0).astype(np.float32)))
    return w, out


def test_pipelined_steps_match_serial_bitwise(ab, cuda):
    w, steps = _steps(5)
    dom = ab.Domain(3, w.periodic, w.radius)
    n = steps[0].shape[0]
    dev = torch.device("cuda:0")
    ctx = ab.Context(0)
    try:
        # serial: copy in, compute, copy out, one stream
        ref = []
        for p in steps:
            pos = torch.from_numpy(p).to(dev)
            E, F, e = ab.lj_energy_forces(ctx, dom, pos, 1.0, 0.01)
            ref.append((E.cpu(), F.cpu(), float(e)))
        # pipelined: two buffers, copies on their own streams
        nb = 2
        hosts = [torch.from_numpy(p).pin_memory() for p in steps]
        pos_d = [torch.empty((n, 3), dtype=torch.float32, device=dev) for _ in range(nb)]
        F_d = [torch.empty((n, 3), dtype=torch.float32, device=dev) for _ in range(nb)]
        E_d = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(nb)]
        e_d = [torch.empty((), dtype=torch.float64, device=dev) for _ in range(nb)]
        F_h = [torch.empty((n, 3), dtype=torch.float32).pin_memory() for _ in steps]
        E_h = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in steps]
        e_h = [torch.empty((), dtype=torch.float64).pin_memory() for _ in steps]
        comp = torch.cuda.current_stream(dev)
        h2d = torch.cuda.Stream(dev)
        d2h = torch.cuda.Stream(dev)
        h2d.wait_stream(comp)
        d2h.wait_stream(comp)
        ev_h, ev_c, ev_d = [], [], []
        for k in range(len(steps)):
            b = k % nb
            ev_h.append(torch.cuda.Event())
            ev_c.append(torch.cuda.Event())
            ev_d.append(torch.cuda.Event())
            with torch.cuda.stream(h2d):
                if k >= nb:
                    h2d.wait_event(ev_c[k - nb])
                pos_d[b].copy_(hosts[k], non_blocking=True)
                ev_h[k].record(h2d)
            comp.wait_event(ev_h[k])
            if k >= nb:
                comp.wait_event(ev_d[k - nb])
            ab.lj_energy_forces(ctx, dom, pos_d[b], 1.0, 0.01, E=E_d[b], F=F_d[b], energy=e_d[b])
            ev_c[k].record(comp)
            with torch.cuda.stream(d2h):
                d2h.wait_event(ev_c[k])
                F_h[k].copy_(F_d[b], non_blocking=True)
                E_h[k].copy_(E_d[b], non_blocking=True)
                e_h[k].copy_(e_d[b], non_blocking=True)
                ev_d[k].record(d2h)
        torch.cuda.synchronize()
        ab.ab_sync(ctx)
        for k, (E, F, e) in enumerate(ref):
            assert torch.equal(E_h[k], E), k
            assert torch.equal(F_h[k], F), k
            assert float(e_h[k]) == e, k
    finally:
        ctx.close()
