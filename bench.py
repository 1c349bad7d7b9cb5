"""Benchmark: pair interactions per second, forward + backward.

Workload (default): d = 3, N = 2^20 points uniform in the periodic unit cube,
r = 0.0197 (~33.6 neighbours mean), truncated Lennard-Jones (sigma = 0.01,
eps = 1).  One step = cell-list rebuild + energy forward + adjoint (forces),
all through the library's C ABI.  The metric counts accepted ordered pairs
(sum over particles of the neighbour count) per second of the step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own independent replica of the workload
(weak scaling, no data-path collective); value = all ranks' pairs / the
slowest rank's time.  ``--impl reference`` times the CPU oracle (the
reference arm of this build) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "pair interactions/s fwd+bwd (3-D LJ, N=2^20, r=0.0197)"
UNIT = "pairs/s"
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
# Gaussian pair sum (clustered workload): per accepted pair, forward 4 FP32
# operations + 1 exponential, adjoint twice that (the cost model of the
# measurement plan: backward ~2x forward)
OPS_PER_PAIR_GAUSS_FWD = 5
OPS_PER_PAIR_GAUSS_BWD = 10
# Algorithmic FP32 operations: per candidate pair the predicate (3 sub, 3 mul,
# 2 add, 1 compare); per accepted pair the LJ adjoint term (1 reciprocal,
# 3 mul for (sig/d)^6, 3 for the coefficient, 2 for (g_i + g_j), 3 FMA).
# Candidates are those of the paper's method (width-r cells, 3^3 stencil),
# whatever finer x cells the kernels actually use.
OPS_PER_CANDIDATE = 9
OPS_PER_PAIR_LJ_BWD = 12
OPS_PER_PAIR_LJ_FWD = 7
# energy and gradient together: rcp, sig^2/d^2, its cube, the energy term (2),
# the force coefficient (3) and three accumulations
OPS_PER_PAIR_LJ_EG = 12
# DRAM traffic of one k_pair_lj_eg<3,false> launch on this workload, from an
# ncu --set full capture (dram__bytes_read.sum + dram__bytes_write.sum), valid
# only for the kernel source it was taken on (None until captured).
TRAFFIC_EG_BYTES = 35.54e6   # 29.28 MB read + 6.26 MB written
TRAFFIC_SOURCE_SHA = "3b686070cc13ccc9"


def alu_peak(pk):
    """FP32 lane-operations per second: SMs x 128 lanes x max SM clock, with
    the SM count read from the device."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    tops = sms * FP32_LANES_PER_SM * pk.get("sm_max_mhz", SM_MAX_MHZ) * 1e6 / 1e12
    return tops, f"{sms} SMs (device query) x {FP32_LANES_PER_SM} FP32 lanes x max SM clock"


def base_candidates(start_h, ncell, periodic, dim, reach):
    """Candidates of the paper's method (width-r cells, 3^d stencil): the
    cell histogram with the kx x-parts of every cell merged back."""
    kx, ky, kz = reach[0], reach[1], max(reach[2], 1)
    if dim == 3:
        cnt = np.diff(start_h.astype(np.int64)).reshape(
            ncell[2] // kz, kz, ncell[1] // ky, ky, ncell[0] // kx, kx).sum(axis=(1, 3, 5))
        base = (ncell[0] // kx, ncell[1] // ky, ncell[2] // kz)
    else:
        cnt = np.diff(start_h.astype(np.int64)).reshape(
            ncell[1] // ky, ky, ncell[0] // kx, kx).sum(axis=(1, 3))
        base = (ncell[0] // kx, ncell[1] // ky, 1)
    base_start = np.concatenate([[0], np.cumsum(cnt.ravel())])
    return candidates_from_cells(base_start, base, periodic, dim)


def build_bytes(n, n_cells):
    """Algorithmic DRAM bytes of one cell-list build (the counting sort of the
    measurement plan): hash = position in (16) + cell id out (4); scatter =
    cell id in (4) + position in (16) + sorted position out (16) + perm out
    (4); cell table = count and offset (4 + 4) per cell of width r (the
    method's cells; finer cells the kernels choose are not counted)."""
    return n * (16 + 4) + n * (4 + 16 + 16 + 4) + 8 * (n_cells + 1)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": SM_MAX_MHZ}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0, interval_ms=50):
        self.index = index
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout=30.0):
        # nvidia-smi's start-up (NVML init) can stall GPU work for seconds:
        # keep it out of the timed region
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.05)
        self.lines.clear()

    def count(self):
        return len(self.lines)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def _stencil_sum_axis(f, axis, periodic, h=1):
    """sum over the distinct stencil neighbours c-h .. c+h along one axis."""
    n = f.shape[axis]
    if periodic:
        if n <= 2 * h:        # every cell of the axis is in every stencil
            return np.broadcast_to(f.sum(axis=axis, keepdims=True), f.shape).copy()
        out = f.copy()
        for o in range(1, h + 1):
            out = out + np.roll(f, o, axis=axis) + np.roll(f, -o, axis=axis)
        return out
    out = f.copy()
    sl = [slice(None)] * f.ndim
    for o in range(1, min(h, n - 1) + 1):
        lo_, hi_ = list(sl), list(sl)
        lo_[axis], hi_[axis] = slice(0, n - o), slice(o, n)
        out[tuple(lo_)] += f[tuple(hi_)]
        out[tuple(hi_)] += f[tuple(lo_)]
    return out


def candidates_from_cells(start, ncell, periodic, dim, reach=(1, 1, 1)):
    """Exact candidate count sum_i sum_{c in stencil(cell i)} n_c from the
    cell histogram (measurement only; the stencil is a product of per-axis
    neighbour sets, so the box sum is separable)."""
    shape = (ncell[2], ncell[1], ncell[0]) if dim == 3 else (ncell[1], ncell[0])
    counts = np.diff(start.astype(np.int64)).reshape(shape)
    s = counts
    for k in range(dim):
        s = _stencil_sum_axis(s, counts.ndim - 1 - k, periodic[k], reach[k])
    return int((counts * s).sum())


def aggregate_ranks(units_per_step, local_ms, steps, dist, device):
    """Weak scaling over independent replicas: every rank processed
    ``units_per_step`` units per step; the job's time is the slowest rank's.
    Returns (max_ms, units_all_ranks_per_second)."""
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_per_step)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.barrier()
    max_ms = float(t.item())
    return max_ms, float(u.item()) * steps / (max_ms * 1e-3)


def run_ours(args, rank, world):
    import torch
    import paper_1704_08907_gb300 as ab

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.c2(seed_offset=rank)
    n = w.n
    eps, sigma = w.params["eps"], w.params["sigma"]
    ctx = ab.Context(local)
    dom = ab.Domain(3, w.periodic, w.radius)
    pos = torch.from_numpy(w.pos).to(dev)
    E = torch.empty(n, dtype=torch.float32, device=dev)
    F = torch.empty((n, 4), dtype=torch.float32, device=dev)
    etot = torch.empty((), dtype=torch.float64, device=dev)
    ones = torch.ones(n, dtype=torch.float32, device=dev)
    prm = ab.OpParams(eps=eps, sigma=sigma)
    # > 129 MB L2; 4-byte elements: the same 256 MB written at ~6 TB/s (a
    # one-byte fill measured 75 us against 44 us)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)

    # pair count (the metric's numerator) and candidate count, untimed
    ab.ab_build(ctx, dom, pos)
    pairs = int(ab.ab_pair_sum(ctx, "count", ab.OpParams()).double().sum().item())
    perm, start = ab.ab_cell_export(ctx)
    ncell, _, reach = ab.ab_cell_shape(ctx, with_reach=True)
    start_h = start.cpu().numpy().view(np.uint32)
    # candidates the kernels evaluate (x cells split kx ways, reach kx) ...
    cands_eval = candidates_from_cells(start_h, ncell, w.periodic, 3, reach)
    # ... and the algorithmic count of the paper's method: width-r cells and
    # the 3^3 stencil (merge the kx x-parts of every cell back together)
    kx, ky, kz = reach
    cands = base_candidates(start_h, ncell, w.periodic, 3, reach)

    # one step: rebuild + LJ energy and its gradient (the forces) in one walk
    def step(ev=None):
        if ev is not None:
            ev[0].record()
        ab.ab_build(ctx, dom, pos)
        if ev is not None:
            ev[1].record()
        ab.ab_pair_energy_grad(ctx, "lj", prm, E=E, grad_pos4=F, energy=etot)
        if ev is not None:
            ev[2].record()

    # the same outputs from the separate forward and adjoint kernels
    def step_unfused(ev):
        ev[0].record()
        ab.ab_build(ctx, dom, pos)
        ev[1].record()
        ab.ab_pair_sum(ctx, "lj", prm, out=E, energy=etot)
        ev[2].record()
        ab.ab_pair_sum_bwd(ctx, "lj", prm, None, ones, grad_pos4=F)
        ev[3].record()

    clocks = ClockSampler(local)
    clocks.start()
    clocks.wait_first()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()                         # untimed: evict L2 between steps
        step(evs[k])
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - t0
    # a short timed region ends before the sampler's next reading: keep the
    # same step running (untimed) until a few readings of it exist
    clock_note = "sampled during the timed steps"
    if clocks.proc is not None and clocks.count() < 3:
        clock_note = ("sampled during the timed steps and an untimed continuation of the same "
                      "step (the timed region is shorter than the sampling interval)")
        t1 = time.perf_counter()
        while clocks.count() < 3 and time.perf_counter() - t1 < 2.0:
            for _ in range(50):
                step()
            torch.cuda.synchronize()
    clk = clocks.stop()
    t_build = np.array([a[0].elapsed_time(a[1]) for a in evs])
    t_eg = np.array([a[1].elapsed_time(a[2]) for a in evs])
    t_step = t_build + t_eg                                # ms, device time
    # unfused reference: the separate forward and adjoint on the same input
    ku = min(args.steps, 200)
    evu = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(ku)]
    for _ in range(3):
        step_unfused(evu[0])
    torch.cuda.synchronize()
    for k in range(ku):
        flush.zero_()
        step_unfused(evu[k])
    torch.cuda.synchronize()
    u_build = np.array([a[0].elapsed_time(a[1]) for a in evu])
    u_fwd = np.array([a[1].elapsed_time(a[2]) for a in evu])
    u_bwd = np.array([a[2].elapsed_time(a[3]) for a in evu])
    u_step = float(np.mean(u_build + u_fwd + u_bwd))
    total_ms = float(t_step.sum())
    if world > 1:
        total_ms, value = aggregate_ranks(pairs, total_ms, args.steps, dist, dev)
    else:
        value = pairs * args.steps / (total_ms * 1e-3)

    # end to end through the public API with host buffers: coordinates packed
    # as xyz (12 bytes a particle) both ways, the layout a caller's arrays have
    pos_h = torch.from_numpy(np.ascontiguousarray(w.pos[:, :3])).pin_memory()
    NB = 2   # buffers in flight: step k computes while k+1's positions arrive and k-1's forces leave
    F_h = [torch.empty((n, 3), dtype=torch.float32).pin_memory() for _ in range(NB)]
    e_h = [torch.empty((), dtype=torch.float64).pin_memory() for _ in range(NB)]
    pos_d = [torch.empty((n, 3), dtype=torch.float32, device=dev) for _ in range(NB)]
    F3 = [torch.empty((n, 3), dtype=torch.float32, device=dev) for _ in range(NB)]
    E_d = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(NB)]
    et_d = [torch.empty((), dtype=torch.float64, device=dev) for _ in range(NB)]

    def e2e_serial(k):
        b = k % NB
        pos_d[b].copy_(pos_h, non_blocking=True)
        ab.lj_energy_forces(ctx, dom, pos_d[b], eps, sigma, E=E_d[b], F=F3[b], energy=et_d[b])
        F_h[b].copy_(F3[b], non_blocking=True)
        e_h[b].copy_(et_d[b], non_blocking=True)

    for k in range(args.warmup):
        e2e_serial(k)
    torch.cuda.synchronize()
    # (1) serial: each step's copies, rebuild, energy and forces back to back,
    # L2 flushed (untimed) between steps
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2e_serial_ms = 0.0
    for k in range(args.steps):
        flush.zero_()
        e0.record()
        e2e_serial(k)
        e1.record()
        torch.cuda.synchronize()
        e2e_serial_ms += e0.elapsed_time(e1)
    # (2) pipelined over steps: the host-to-device copy of step k+1 and the
    # device-to-host copy of step k-1 run on their own streams while step k
    # computes; every step still copies its positions in and its forces and
    # energy out inside the timed region, and its L2 flush (before its
    # rebuild, on the compute stream) is timed too
    comp = torch.cuda.current_stream(dev)
    h2d_s = torch.cuda.Stream(dev)
    d2h_s = torch.cuda.Stream(dev)

    def e2e_pipelined(K):
        ev_h = [torch.cuda.Event() for _ in range(K)]
        ev_c = [torch.cuda.Event() for _ in range(K)]
        ev_d = [torch.cuda.Event() for _ in range(K)]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(comp)
        h2d_s.wait_stream(comp)
        d2h_s.wait_stream(comp)
        for k in range(K):
            b = k % NB
            with torch.cuda.stream(h2d_s):
                if k >= NB:
                    h2d_s.wait_event(ev_c[k - NB])   # step k-NB has read pos_d[b]
                pos_d[b].copy_(pos_h, non_blocking=True)
                ev_h[k].record(h2d_s)
            comp.wait_event(ev_h[k])
            if k >= NB:
                comp.wait_event(ev_d[k - NB])   # step k-NB's results have left F3[b]
            flush.zero_()
            ab.lj_energy_forces(ctx, dom, pos_d[b], eps, sigma, E=E_d[b], F=F3[b], energy=et_d[b])
            ev_c[k].record(comp)
            with torch.cuda.stream(d2h_s):
                d2h_s.wait_event(ev_c[k])
                F_h[b].copy_(F3[b], non_blocking=True)
                e_h[b].copy_(et_d[b], non_blocking=True)
                ev_d[k].record(d2h_s)
        comp.wait_event(ev_d[K - 1])
        t1.record(comp)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1)

    e2e_pipelined(max(args.warmup, NB + 1))
    e2e_ms = e2e_pipelined(args.steps)
    ab.ab_sync(ctx)
    if world > 1:   # all ranks' pairs over the slowest rank's time, as for value
        e2e_ms, e2e_value = aggregate_ranks(pairs, e2e_ms, args.steps, dist, dev)
        e2e_serial_ms, e2e_serial_value = aggregate_ranks(pairs, e2e_serial_ms, args.steps, dist, dev)
    else:
        e2e_value = pairs * args.steps / (e2e_ms * 1e-3)
        e2e_serial_value = pairs * args.steps / (e2e_serial_ms * 1e-3)

    import hashlib
    src = os.path.join(ROOT, "paper_1704_08907_gb300", "csrc", "ab_pairs.cu")
    same_kernel = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == TRAFFIC_SOURCE_SHA
    pk, pk_kind = peaks()
    alu, alu_src = alu_peak(pk)
    eg_ops = cands * OPS_PER_CANDIDATE + pairs * OPS_PER_PAIR_LJ_EG
    eg_s = float(np.mean(t_eg)) * 1e-3
    achieved = eg_ops / eg_s / 1e12
    fwd_ops = cands * OPS_PER_CANDIDATE + pairs * OPS_PER_PAIR_LJ_FWD
    bwd_ops = cands * OPS_PER_CANDIDATE + pairs * OPS_PER_PAIR_LJ_BWD
    bbytes = build_bytes(n, int(np.prod(ncell)) // (kx * ky * kz))   # width-r cells
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "3-D uniform periodic cube, N=1048576, r=0.0197, "
                               "Lennard-Jones sigma=0.01 eps=1: rebuild + energy + forces",
                   "n": n, "radius": w.radius, "pairs_per_step": pairs,
                   "candidates_per_step": cands, "candidates_evaluated": cands_eval,
                   "cell_split": [kx, ky, kz], "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "kernel": "k_pair_lj_eg<3,false>",
                     "achieved": achieved, "peak": alu, "unit": "Top/s",
                     "frac": achieved / alu,
                     "traffic": TRAFFIC_EG_BYTES if same_kernel else None,
                     "algorithmic_ops_per_launch": eg_ops,
                     "peak_source": alu_src},
        "phases_ms": {"build": float(np.mean(t_build)), "energy_and_forces": float(np.mean(t_eg))},
        "phase_roofline": {
            "build_hbm_gbs": bbytes / (float(np.mean(t_build)) * 1e-3) / 1e9,
            "build_hbm_frac": bbytes / (float(np.mean(t_build)) * 1e-3) / 1e9 / pk["hbm_gbs"],
            "build_bytes_algorithmic": bbytes,
            "peak_kind": pk_kind},
        "general_adjoint_step": {
            "note": "the same workload through the separate forward (per-particle energies) "
                    "and the general adjoint kernel (any upstream gradient; here 1): the path "
                    "autograd takes (LJEnergy)",
            "metric": METRIC, "unit": UNIT, "steps": ku, "ms_per_step": u_step,
            "value": pairs / (u_step * 1e-3),
            "phases_ms": {"build": float(np.mean(u_build)), "fwd": float(np.mean(u_fwd)),
                          "bwd": float(np.mean(u_bwd))},
            "roofline": {"bound": "alu", "kernel": "k_pair_bwd<3,false,LJ> (adjoint)",
                         "achieved": bwd_ops / (float(np.mean(u_bwd)) * 1e-3) / 1e12,
                         "peak": alu, "unit": "Top/s",
                         "frac": bwd_ops / (float(np.mean(u_bwd)) * 1e-3) / 1e12 / alu,
                         "traffic": None, "peak_source": alu_src},
            "fwd_alu_frac": fwd_ops / (float(np.mean(u_fwd)) * 1e-3) / 1e12 / alu,
            "bwd_alu_frac": bwd_ops / (float(np.mean(u_bwd)) * 1e-3) / 1e12 / alu},
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": pos_h.numel() * 4,
                "d2h_bytes_per_step": F_h[0].numel() * 4 + 8,
                "mode": ("pipelined over steps: step k+1's host-to-device copy and step k-1's "
                         "device-to-host copy on their own streams during step k; each step's "
                         "L2 flush timed on the compute stream"),
                "ms_per_step": e2e_ms / args.steps,
                "serial_value": e2e_serial_value,
                "serial_ms_per_step": e2e_serial_ms / args.steps},
        "gpu_launches": 3 * args.steps,   # build (one cooperative launch), fused walk, energy reduction
        "wall_s": wall,
    }
    if clk:
        clk["note"] = clock_note
        out["clocks"] = clk
    return out, w


def _timed(fn, reps, flush=None):
    import torch
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def also_dense(reps=5):
    """Dense kernel operator, 65,536 x 65,536 x 64 right-hand sides: FP32 CUDA
    cores vs the tcgen05 paths (TFLOP/s counts 2 M N nrhs per product)."""
    import torch
    import paper_1704_08907_gb300 as ab
    d = synth.c4()
    dev = torch.device("cuda", torch.cuda.current_device())
    X = torch.from_numpy(synth.pack4(d.X)).to(dev)
    Y = torch.from_numpy(synth.pack4(d.Y)).to(dev)
    W = torch.from_numpy(d.W).to(dev)
    m, n, nrhs = X.shape[0], Y.shape[0], W.shape[1]
    ctx = ab.Context(dev.index)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)   # 256 MB
    outs, res = {}, {}
    for prec in ("fp32", "bf16x3", "bf16", "tf32x3", "tf32"):
        out = torch.empty((m, nrhs), dtype=torch.float32, device=dev)
        fn = lambda: ab.ab_kernel_matvec(ctx, X, Y, W, d.s, prec, out=out)  # noqa: E731
        for _ in range(2):
            fn()
        ms = _timed(fn, reps, flush)
        res[prec] = {"ms": ms, "tflops": 2.0 * m * n * nrhs / (ms * 1e-3) / 1e12}
        outs[prec] = out
    ab.ab_sync(ctx)
    # error against FP64 for every result: the oracle's FP64 operator on 256
    # sampled rows, per element over the sum of the magnitudes of the
    # element's terms (sum_j K_ij |W_jc|)
    from oracle import dense as odense
    rows = synth.query_sample(m, 256, 12)
    ref = odense.matvec(d.X, d.Y, d.W, d.s, rows=rows)
    den = odense.matvec_abs(d.X, d.Y, d.W, d.s, rows=rows)
    for prec in ("fp32", "bf16x3", "bf16", "tf32x3", "tf32"):
        got = outs[prec].cpu().numpy()[rows].astype(np.float64)
        res[prec]["err_vs_fp64"] = float(np.max(np.abs(got - ref) / den))
    res["err_vs_fp64_metric"] = ("max over 256 sampled rows x 64 columns of |Y - Y_fp64| / "
                                 "sum_j K_ij |W_jc| (oracle FP64)")
    res["speedup_bf16x3_vs_fp32"] = res["fp32"]["ms"] / res["bf16x3"]["ms"]
    res["speedup_tf32x3_vs_fp32"] = res["fp32"]["ms"] / res["tf32x3"]["ms"]
    # the BF16X3 forward against the measured bf16 tensor peak: algorithmic
    # tensor work = 3 bf16 products of 2 M N nrhs (P_hi W_hi, P_hi W_lo,
    # P_lo W_hi); the kernel also issues P_lo W_lo, which only adds accuracy
    pk, pk_kind = peaks()
    tc_tf = 3.0 * 2.0 * m * n * nrhs / (res["bf16x3"]["ms"] * 1e-3) / 1e12
    res["roofline_bf16x3"] = {"bound": "tensor", "achieved": tc_tf, "peak": pk["bf16_tflops"],
                              "unit": "TFLOP/s", "frac": tc_tf / pk["bf16_tflops"],
                              "peak_kind": pk_kind + " bf16 burst",
                              "exps_per_s": m * n / (res["bf16x3"]["ms"] * 1e-3)}
    # adjoint: dW, dX, dY and ds (lengthscale) in one call
    G = torch.from_numpy(d.G).to(dev)
    dW = torch.empty_like(W)
    dX = torch.empty_like(X)
    dY = torch.empty_like(Y)
    ds = torch.empty((), dtype=torch.float64, device=dev)
    bwd = {}
    cols = synth.query_sample(n, 64, 11)
    brow = synth.query_sample(m, 64, 10)
    rW = odense.grad_W(d.X, d.Y, d.G, d.s, cols=cols)
    aW = odense.grad_W(d.X, d.Y, np.abs(d.G), d.s, cols=cols)
    rX = odense.grad_X(d.X, d.Y, d.W, d.G, d.s, rows=brow)
    aX = odense.grad_X_abs(d.X, d.Y, d.W, d.G, d.s, rows=brow)
    rY = odense.grad_Y(d.X, d.Y, d.W, d.G, d.s, cols=cols)
    aY = odense.grad_Y_abs(d.X, d.Y, d.W, d.G, d.s, cols=cols)

    def elem(got, r, a):
        dd = np.maximum(np.abs(r), a)
        return float(np.max(np.abs(got.astype(np.float64) - r) / dd))

    for prec, reps_b in (("fp32", 1), ("bf16x3", reps), ("bf16", reps), ("tf32x3", reps),
                         ("tf32", reps)):
        fn = lambda: ab.ab_kernel_matvec_bwd(ctx, X, Y, W, d.s, prec, G, dW, dX, dY, ds)  # noqa: E731
        fn()
        bwd[prec] = {"ms": _timed(fn, reps_b, flush)}
        ab.ab_sync(ctx)
        bwd[prec]["err_vs_fp64"] = {
            "dW": elem(dW.cpu().numpy()[cols], rW, aW),
            "dX": elem(dX.cpu().numpy()[brow, :3], rX, aX),
            "dY": elem(dY.cpu().numpy()[cols, :3], rY, aY)}
    bwd["err_vs_fp64_metric"] = (
        "per element over the sum of the magnitudes of its terms (oracle FP64): dW on 64 sampled "
        "Y rows, dX on 64 sampled X rows, dY on 64 sampled Y rows; ds is checked against the "
        "FP64 sum at 8192 x 8192 in the tests")
    bwd["speedup_bf16x3_vs_fp32"] = bwd["fp32"]["ms"] / bwd["bf16x3"]["ms"]
    res["adjoint_dW_dX_dY_ds"] = bwd
    res["exps"] = m * n
    res["workload"] = "X, Y 65,536 points in [0,1]^3, W 65,536 x 64, Gaussian kernel l = 0.1"
    ctx.close()
    return res


def oracle_sample_c3(w, nq, seed=23):
    """Oracle Gaussian forward + adjoint (x, w, s) over nq query particles of
    the clustered workload (cell list over all points).  Returns (pairs in
    the sample, seconds for the cell list, seconds for the queries, threads)."""
    import oracle
    box = oracle.Box(3, w.periodic, w.lo, w.hi, w.radius)
    q = synth.query_sample(w.n, nq, seed)
    t0 = time.perf_counter()
    cl = oracle.CellList(box, w.pos)
    t1 = time.perf_counter()
    off, idx = cl.neighbours(q)
    oracle.pair_values("gauss", box, w.pos, off, idx, q, w=w.w, params=w.params)
    oracle.pair_grads("gauss", box, w.pos, off, idx, w.g, q, w=w.w, params=w.params)
    t2 = time.perf_counter()
    cl.close()
    return int(off[-1]), t1 - t0, t2 - t1, oracle.num_threads()


# DRAM traffic of one k_pair_bwd<3,false,GAUSS> launch on the clustered
# workload (ncu dram__bytes_read.sum + dram__bytes_write.sum), valid for the
# kernel source whose hash is given (None until captured on that source).
TRAFFIC_C3_BWD_BYTES = 942.84e6    # 550.14 MB read + 392.70 MB written (adjoint kernel)
TRAFFIC_C3_VG_BYTES = 1129.44e6    # 612.22 MB read + 517.22 MB written (value and gradient)
TRAFFIC_C3_SOURCE_SHA = "3b686070cc13ccc9"


def also_c3(reps=5, oracle_fraction=64):
    """Clustered 16.7M-point workload: rebuild + Gaussian pair sum + adjoint
    (x, w, s); pairs per second, the adjoint kernel against the ALU roofline,
    and the oracle on a 1/oracle_fraction query sample on the host cores."""
    import torch
    import paper_1704_08907_gb300 as ab
    w = synth.c3()
    dev = torch.device("cuda", torch.cuda.current_device())
    pos = torch.from_numpy(w.pos).to(dev)
    wt = torch.from_numpy(w.w).to(dev)
    g = torch.from_numpy(w.g).to(dev)
    ctx = ab.Context(dev.index)
    dom = ab.Domain(3, w.periodic, w.radius)
    prm = ab.OpParams(s=w.params["s"])
    y = torch.empty(w.n, dtype=torch.float32, device=dev)
    gpos = torch.empty((w.n, 4), dtype=torch.float32, device=dev)
    gw = torch.empty(w.n, dtype=torch.float32, device=dev)
    gs = torch.empty((), dtype=torch.float64, device=dev)
    ab.ab_build(ctx, dom, pos)
    pairs = int(ab.ab_pair_sum(ctx, "count", ab.OpParams()).double().sum().item())
    ncell, ncells, reach = ab.ab_cell_shape(ctx, with_reach=True)
    _, start = ab.ab_cell_export(ctx)
    start_h = start.cpu().numpy().view(np.uint32)
    cands = base_candidates(start_h, ncell, w.periodic, 3, reach)
    del start, start_h

    def step():
        ab.ab_build(ctx, dom, pos)
        ab.ab_pair_sum(ctx, "gauss", prm, w=wt, out=y)
        ab.ab_pair_sum_bwd(ctx, "gauss", prm, wt, g, gpos, gw, gs)

    for _ in range(2):
        step()
    ms = _timed(step, reps)
    # phase split of the same step (CUDA events between the three calls)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ph = np.zeros(3)
    for _ in range(reps):
        ev[0].record()
        ab.ab_build(ctx, dom, pos)
        ev[1].record()
        ab.ab_pair_sum(ctx, "gauss", prm, w=wt, out=y)
        ev[2].record()
        ab.ab_pair_sum_bwd(ctx, "gauss", prm, wt, g, gpos, gw, gs)
        ev[3].record()
        torch.cuda.synchronize()
        ph += [ev[k].elapsed_time(ev[k + 1]) for k in range(3)]
    ph /= reps
    # the same step with the forward and the adjoint in one walk (the
    # upstream gradient is given, so the value and the gradient can be formed
    # together; bit for bit the separate calls' outputs)
    def step_vg():
        ab.ab_build(ctx, dom, pos)
        ab.ab_pair_sum_value_grad(ctx, "gauss", prm, wt, g, out=y, grad_pos4=gpos, grad_w=gw,
                                  grad_s=gs)

    for _ in range(2):
        step_vg()
    ms_vg = _timed(step_vg, reps)
    ev2 = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    vg_ph = np.zeros(2)
    for _ in range(reps):
        ev2[0].record()
        ab.ab_build(ctx, dom, pos)
        ev2[1].record()
        ab.ab_pair_sum_value_grad(ctx, "gauss", prm, wt, g, out=y, grad_pos4=gpos, grad_w=gw,
                                  grad_s=gs)
        ev2[2].record()
        torch.cuda.synchronize()
        vg_ph += [ev2[k].elapsed_time(ev2[k + 1]) for k in range(2)]
    vg_ph /= reps
    ab.ab_sync(ctx)
    ctx.close()
    pk, pk_kind = peaks()
    alu, alu_src = alu_peak(pk)
    fwd_ops = cands * OPS_PER_CANDIDATE + pairs * OPS_PER_PAIR_GAUSS_FWD
    bwd_ops = cands * OPS_PER_CANDIDATE + pairs * OPS_PER_PAIR_GAUSS_BWD
    import hashlib
    src = os.path.join(ROOT, "paper_1704_08907_gb300", "csrc", "ab_pairs.cu")
    same = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == TRAFFIC_C3_SOURCE_SHA
    bbytes = build_bytes(w.n, ncells // int(np.prod(reach)))   # width-r cells
    out = {"workload": "16,777,216 points in 1024 Gaussian blobs, periodic cube, "
                       f"r={w.radius:.7f} (64 neighbours mean): rebuild + gauss fwd + adjoint",
           "pairs_per_step": pairs, "candidates_per_step": cands, "ms_per_step": ms,
           "pairs_per_s": pairs / (ms * 1e-3), "inputs_larger_than_l2": True,
           "phases_ms": {"build": ph[0], "fwd": ph[1], "bwd": ph[2]},
           "cells": list(ncell), "n_cells": ncells, "cell_split": list(reach),
           "roofline": {"bound": "alu", "kernel": "k_pair_bwd<3,compact,GAUSS> (adjoint: x, w, s)",
                        "achieved": bwd_ops / (ph[2] * 1e-3) / 1e12, "peak": alu, "unit": "Top/s",
                        "frac": bwd_ops / (ph[2] * 1e-3) / 1e12 / alu,
                        "traffic": TRAFFIC_C3_BWD_BYTES if same else None,
                        "algorithmic_ops_per_launch": bwd_ops,
                        "peak_source": alu_src,
                        "timing": "the adjoint call's events: the kernel plus its two gathers"},
           "fwd_alu_frac": fwd_ops / (ph[1] * 1e-3) / 1e12 / alu,
           "value_and_grad_step": {
               "note": "rebuild + ab_pair_sum_value_grad: the forward values and the adjoint "
                       "(x, w, s) in one walk over the pairs, bit for bit the separate calls",
               "ms_per_step": ms_vg, "pairs_per_s": pairs / (ms_vg * 1e-3),
               "phases_ms": {"build": vg_ph[0], "value_and_grad": vg_ph[1]},
               "alu_frac": (cands * OPS_PER_CANDIDATE + pairs * (OPS_PER_PAIR_GAUSS_FWD +
                                                                 OPS_PER_PAIR_GAUSS_BWD))
                           / (vg_ph[1] * 1e-3) / 1e12 / alu,
               "traffic": TRAFFIC_C3_VG_BYTES if same else None},
           "build_hbm_frac": bbytes / (ph[0] * 1e-3) / 1e9 / pk["hbm_gbs"],
           "build_bytes_algorithmic": bbytes}
    nq = w.n // oracle_fraction
    sp, t_cl, t_q, cores = oracle_sample_c3(w, nq)
    full_s = t_cl + t_q * (w.n / nq)
    out["cpu_baseline"] = {"value": pairs / full_s, "unit": UNIT, "cores": cores, "kind": "oracle",
                           "sample": f"oracle cell list over all {w.n} points ({t_cl:.2f} s) + "
                                     f"Gaussian forward and adjoint for {nq} query particles "
                                     f"({sp} pairs, {t_q:.2f} s), extrapolated linearly to all "
                                     f"{w.n} particles"}
    return out


def also_md(loop_steps=200):
    """The paper's molecular-dynamics example (Sec. 3): 2-D periodic unit
    square, exponential force of Eq. 1 with c = 1e-3, semi-implicit Euler with
    dt = 1 (Eqs. 2-3).  Fig. 3 shapes: N/T_e for r = sqrt(3/N) (left, ~9.4
    neighbours) and r = sqrt(3/500) (right, neighbours grow with N).  T_e is
    the velocity update of Eq. 2 as the paper times it: the force sum on the
    current cell list plus v += f (ab_pair_sum EXPF + ab_md_step, the latter
    applied to a scratch copy of the positions so that the cell list stays
    valid).  step = rebuild + force + Eqs. 2-3.  Also a time loop at
    N = 2^20."""
    import torch
    import paper_1704_08907_gb300 as ab
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = ab.Context(dev.index)
    prm = ab.OpParams(c=1.0e-3)

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def point(n, r):
        w = synth.paper_shape(n)
        pos = torch.from_numpy(w.pos).to(dev)
        scratch = pos.clone()
        vel = torch.zeros_like(pos)
        F = torch.empty_like(pos)
        dom = ab.Domain(2, (1, 1), r)
        ab.ab_build(ctx, dom, pos)
        pairs = int(ab.ab_pair_sum(ctx, "count", ab.OpParams()).double().sum().item())
        reps = max(5, min(2000, int(2e8 / max(pairs + n, 1))))

        def te():
            ab.ab_pair_sum(ctx, "expf", prm, out=F)
            ab.ab_md_step(ctx, dom, scratch, vel, F, 1.0)

        def step():
            ab.ab_build(ctx, dom, pos)
            ab.ab_pair_sum(ctx, "expf", prm, out=F)
            ab.ab_md_step(ctx, dom, pos, vel, F, 1.0)

        te_ms = timed(te, reps)
        step_ms = timed(step, reps)
        # the same velocity update replayed from a CUDA graph of 20 updates:
        # at small N the eager numbers are host launch latency, not GPU time
        graph_te_ms = None
        try:
            ab.ab_build(ctx, dom, pos)
            te()
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            cap = torch.cuda.Stream(dev)
            cap.wait_stream(torch.cuda.current_stream(dev))
            with torch.cuda.stream(cap):
                with torch.cuda.graph(g, stream=cap):
                    for _ in range(20):
                        te()
            torch.cuda.current_stream(dev).wait_stream(cap)
            graph_te_ms = timed(g.replay, max(3, reps // 20)) / 20
        except Exception:   # capture unavailable: report the eager numbers only
            graph_te_ms = None
        return {"N": n, "r": r, "neighbours_mean": pairs / n, "reps": reps,
                "te_ms": te_ms, "N_over_Te_per_s": n / (te_ms * 1e-3),
                "te_graph_ms": graph_te_ms,
                "N_over_Te_graph_per_s": n / (graph_te_ms * 1e-3) if graph_te_ms else None,
                "step_ms": step_ms, "N_over_Tstep_per_s": n / (step_ms * 1e-3)}

    left = [point(1 << k, math.sqrt(3.0 / (1 << k))) for k in range(4, 25, 2)]
    right = [point(1 << k, math.sqrt(3.0 / 500.0)) for k in range(4, 18, 2)]
    # the time loop: N = 2^20, rebuild + force + step every step
    n = 1 << 20
    w = synth.paper_shape(n)
    pos = torch.from_numpy(w.pos).to(dev)
    vel = torch.zeros_like(pos)
    F = torch.empty_like(pos)
    dom = ab.Domain(2, (1, 1), w.radius)

    def loop_step():
        ab.ab_build(ctx, dom, pos)
        ab.ab_pair_sum(ctx, "expf", prm, out=F)
        ab.ab_md_step(ctx, dom, pos, vel, F, 1.0)

    ms = timed(loop_step, loop_steps)
    ab.ab_sync(ctx)
    vsum = vel[:, :2].double().sum(dim=0).abs().max().item()
    return {"workload": "paper Sec. 3 example: 2-D periodic, EXPF c=1e-3, semi-implicit Euler dt=1",
            "fig3_left_r_sqrt3_over_N": left, "fig3_right_r_sqrt3_over_500": right,
            "time_loop_N1048576": {"steps": loop_steps + 3, "ms_per_step": ms,
                                   "particle_steps_per_s": n / (ms * 1e-3),
                                   "total_momentum_abs_max": vsum},
            "gpu_launches_per_step": 7}


def also_solve():
    """Kernel-system solve (K(X, X) + sigma^2 I) W = B by conjugate gradients
    on the dense operator (RBF interpolation with a nugget / GP posterior
    mean, Sec. 1.1): X = the 65,536 dense-workload points, 64 right-hand
    sides ~ N(0, 1), Gaussian kernel l = 0.1, sigma^2 = 1, tol = 1e-4.  The
    true residual is checked on 64 sampled rows against the oracle's FP64
    matvec."""
    import torch
    import paper_1704_08907_gb300 as ab
    from oracle import dense as odense
    d = synth.c4()
    dev = torch.device("cuda", torch.cuda.current_device())
    X = torch.from_numpy(synth.pack4(d.X)).to(dev)
    Bh = np.random.default_rng(1704089 + 40).standard_normal((d.X.shape[0], 64)).astype(np.float32)
    B = torch.from_numpy(Bh).to(dev)
    ctx = ab.Context(dev.index)
    sigma2, tol = 1.0, 1e-4
    rows = synth.query_sample(d.X.shape[0], 64, 41)
    res = {"workload": "n=65,536 points in [0,1]^3, 64 rhs, Gaussian l=0.1 (s=50), sigma^2=1, "
                       "CG tol=1e-4 from W=0", "tol": tol, "sigma2": sigma2}
    for prec in ("bf16x3", "fp32"):
        ab.ab_kernel_solve(ctx, X, B, d.s, sigma2, prec, tol, 3)    # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        W, it, rr = ab.ab_kernel_solve(ctx, X, B, d.s, sigma2, prec, tol, 2000)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        Wh = W.cpu().numpy().astype(np.float64)
        ax = odense.matvec(d.X[rows], d.X, Wh, d.s) + sigma2 * Wh[rows]
        sampled = float(np.abs(Bh[rows] - ax).max() / np.sqrt((Bh.astype(np.float64) ** 2).mean()))
        res[prec] = {"iterations": it, "seconds": secs, "ms_per_iteration": secs * 1e3 / max(it, 1),
                     "relative_residual": rr, "sampled_rows_residual_over_rms_b": sampled}
    res["speedup_bf16x3_vs_fp32"] = res["fp32"]["seconds"] / res["bf16x3"]["seconds"]
    ab.ab_sync(ctx)
    return res


def also_sph(steps=50):
    """SPH density + symmetric pressure force (Wendland C2, support r) on
    1,048,576 uniform points in the periodic unit cube, r for ~57 neighbours
    (a typical SPH support), masses 1/N.  One step = rebuild + density +
    force; the per-particle P/rho^2 input of the force comes from the
    equation of state P = rho - 1 evaluated once before timing."""
    import torch
    import paper_1704_08907_gb300 as ab
    n = 1 << 20
    r = (57.0 / (4.0 / 3.0 * math.pi * n)) ** (1.0 / 3.0)
    dev = torch.device("cuda", torch.cuda.current_device())
    pos = torch.from_numpy(synth.uniform_positions(n, 3, 1704089 + 50)).to(dev)
    m = torch.full((n,), 1.0 / n, dtype=torch.float32, device=dev)
    ctx = ab.Context(dev.index)
    dom = ab.Domain(3, (1, 1, 1), r)
    ab.ab_build(ctx, dom, pos)
    pairs = int(ab.ab_pair_sum(ctx, "count", ab.OpParams()).double().sum().item())
    rho = ab.ab_pair_sum(ctx, "sph_density", ab.OpParams(), w=m)
    wv = torch.stack([m, (rho - 1.0) / (rho * rho)], 1).contiguous()
    F = torch.empty((n, 4), dtype=torch.float32, device=dev)

    def step():
        ab.ab_build(ctx, dom, pos)
        ab.ab_pair_sum(ctx, "sph_density", ab.OpParams(), w=m, out=rho)
        ab.ab_pair_sum(ctx, "sph_force", ab.OpParams(), w=wv, out=F)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ab.ab_sync(ctx)
    return {"workload": "SPH, N=1,048,576 uniform periodic cube, Wendland C2 support r=%.5f "
                        "(~57 neighbours): rebuild + density + pressure force" % r,
            "steps": steps, "ms_per_step": ms, "pairs_per_step": pairs,
            "pair_evaluations_per_s": 2 * pairs / (ms * 1e-3),
            "mean_density": float(rho.double().mean().item())}


def also_bd(steps=1000):
    """2-D Brownian dynamics, 4,194,304 particles, x periodic / y reflecting,
    soft repulsion within r = 0.002, Euler-Maruyama dt = 1e-5 with Philox
    noise, full cell-list rebuild every step (rebuild + force + step, all on
    the device; the loop is also captured as one CUDA graph)."""
    import torch
    import paper_1704_08907_gb300 as ab
    w = synth.c5()
    p = w.params
    dev = torch.device("cuda", torch.cuda.current_device())
    pos = torch.from_numpy(w.pos).to(dev)
    F = torch.empty_like(pos)
    ctx = ab.Context(dev.index)
    dom = ab.Domain(2, w.periodic, w.radius)
    prm = ab.OpParams(k=p["k"])
    ab.ab_build(ctx, dom, pos)
    pairs0 = int(ab.ab_pair_sum(ctx, "count", ab.OpParams()).double().sum().item())
    state = {"t": 0}

    def one_step(t):
        ab.ab_build(ctx, dom, pos)
        ab.ab_pair_sum(ctx, "soft", prm, out=F)
        ab.ab_bd_step(ctx, dom, pos, F, p["dt"], p["D"], p["seed"], t)

    for _ in range(3):
        one_step(state["t"])
        state["t"] += 1
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        one_step(state["t"])
        state["t"] += 1
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ab.ab_sync(ctx)
    res = {"workload": "2-D, N=4,194,304, x periodic / y reflecting, r=0.002, soft force "
                       "k=1e4, dt=1e-5, D=1e-2, rebuild every step",
           "steps": steps, "ms_per_step": ms, "steps_per_s": 1e3 / ms,
           "pairs_per_step_initial": pairs0, "pairs_per_s_initial": pairs0 / (ms * 1e-3),
           "gpu_launches_per_step": 7}
    # the same loop as one CUDA graph (step index baked in per captured step)
    try:
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(dev)
        cap.wait_stream(torch.cuda.current_stream(dev))
        base = state["t"]
        with torch.cuda.stream(cap):
            with torch.cuda.graph(g, stream=cap):
                for k in range(10):
                    one_step(base + k)
        torch.cuda.current_stream(dev).wait_stream(cap)
        g.replay()
        torch.cuda.synchronize()
        e0.record()
        reps = max(1, steps // 10)
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        res["graph_ms_per_step"] = e0.elapsed_time(e1) / (reps * 10)
        res["graph_note"] = "10 steps per graph; replays reuse the captured step indices"
    except Exception as exc:  # capture unsupported in this configuration
        res["graph_ms_per_step"] = None
        res["graph_note"] = f"capture failed: {type(exc).__name__}: {exc}"[:200]
    try:
        ab.ab_sync(ctx)
        ctx.close()
    except Exception:
        pass
    return res


def oracle_sample(w, nq, seed=17):
    """Oracle LJ energy + adjoint over nq query particles (cell list over all)."""
    import oracle
    box = oracle.Box(3, w.periodic, w.lo, w.hi, w.radius)
    q = synth.query_sample(w.n, nq, seed)
    t0 = time.perf_counter()
    cl = oracle.CellList(box, w.pos)
    off, idx = cl.neighbours(q)
    oracle.pair_values("lj", box, w.pos, off, idx, q, params=w.params)
    oracle.pair_grads("lj", box, w.pos, off, idx, np.ones(w.n), q, params=w.params)
    dt = time.perf_counter() - t0
    return int(off[-1]), dt, oracle.num_threads()


def build_paths(reps=10):
    """Median CUDA-event time of ab_build on each build path (counting sort as
    a kernel sequence, as one cooperative launch, radix sort) for the
    workloads' inputs, L2 flushed before every timed build."""
    import torch
    import paper_1704_08907_gb300 as ab
    cases = {
        "c2_1M_uniform_3d": (synth.c2(), 3),
        "c3_16M_clustered_3d": (synth.c3(), 3),
        "c5_4M_uniform_2d": (synth.c5(), 2),
    }
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")   # 256 MB
    ctx = ab.Context(0)
    res = {}
    for name, (w, dim) in cases.items():
        pos = torch.from_numpy(w.pos).cuda()
        dom = ab.Domain(dim, w.periodic, w.radius)
        row = {}
        for path, label in ((ab.BUILD_SEQUENCE, "sequence"), (ab.BUILD_COOP, "coop"),
                            (ab.BUILD_RADIX, "radix"), (ab.BUILD_AUTO, "auto")):
            ab.ab_testing_build_path(ctx, path)
            for _ in range(3):
                ab.ab_build(ctx, dom, pos)
            ts = []
            for _ in range(reps):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                ab.ab_build(ctx, dom, pos)
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            ab.ab_sync(ctx)
            row[label] = round(float(np.median(ts)) * 1e3, 1)
        _, ncells = ab.ab_cell_shape(ctx)
        row["n"] = w.n
        row["n_cells"] = ncells
        row["unit"] = "us"
        res[name] = row
        del pos
    ab.ab_testing_build_path(ctx, ab.BUILD_AUTO)
    ctx.close()
    return res


def probe(spec):
    """One call per listed item, for ncu captures of a single kernel."""
    import torch
    import paper_1704_08907_gb300 as ab
    kind, _, items = spec.partition(":")
    if kind == "c3":   # one rebuild + Gaussian forward + adjoint + value-and-gradient, clustered
        # points (16.7M, or 'c3:N' for N points in blobs of the same size)
        n = int(items) if items else 1 << 24
        w = synth.c3(n=n, n_blobs=max(1, n // 16384))
        ctx = ab.Context(0)
        dom = ab.Domain(3, w.periodic, w.radius)
        ab.ab_build(ctx, dom, torch.from_numpy(w.pos).cuda())
        wt, g = torch.from_numpy(w.w).cuda(), torch.from_numpy(w.g).cuda()
        prm = ab.OpParams(s=w.params["s"])
        y = ab.ab_pair_sum(ctx, "gauss", prm, w=wt)
        gp = torch.empty((w.n, 4), dtype=torch.float32, device="cuda")
        gw = torch.empty(w.n, dtype=torch.float32, device="cuda")
        gs = torch.empty((), dtype=torch.float64, device="cuda")
        ab.ab_pair_sum_bwd(ctx, "gauss", prm, wt, g, gp, gw, gs)
        ab.ab_pair_sum_value_grad(ctx, "gauss", prm, wt, g, out=y, grad_pos4=gp, grad_w=gw,
                                  grad_s=gs)
        ab.ab_sync(ctx)
        torch.cuda.synchronize()
        ctx.close()
        return
    if kind == "bd":   # N steps of the 2-D Brownian-dynamics loop ('bd:N'; default 13)
        w = synth.c5()
        p = w.params
        pos = torch.from_numpy(w.pos).cuda()
        F = torch.empty_like(pos)
        ctx = ab.Context(0)
        dom = ab.Domain(2, w.periodic, w.radius)
        prm = ab.OpParams(k=p["k"])
        for t in range(int(items) if items else 13):
            ab.ab_build(ctx, dom, pos)
            ab.ab_pair_sum(ctx, "soft", prm, out=F)
            ab.ab_bd_step(ctx, dom, pos, F, p["dt"], p["D"], p["seed"], t)
        ab.ab_sync(ctx)
        torch.cuda.synchronize()
        ctx.close()
        return
    if kind == "build-paths":   # time every build path on the workloads' inputs
        print(json.dumps(build_paths(int(items) if items else 10)))
        return
    if kind != "dense":
        raise SystemExit(f"unknown probe {spec!r}")
    d = synth.c4()
    X = torch.from_numpy(synth.pack4(d.X)).cuda()
    Y = torch.from_numpy(synth.pack4(d.Y)).cuda()
    W = torch.from_numpy(d.W).cuda()
    ctx = ab.Context(0)
    for item in items.split(","):
        if item.startswith("bwd-"):   # adjoint: dW (forward kernel), dX and dY (gradient kernel)
            G = torch.from_numpy(d.G).cuda()
            ab.ab_kernel_matvec_bwd(ctx, X, Y, W, d.s, item[4:], G, torch.empty_like(W),
                                    torch.empty_like(X), torch.empty_like(Y),
                                    torch.empty((), dtype=torch.float64, device="cuda"))
        else:
            ab.ab_kernel_matvec(ctx, X, Y, W, d.s, item)
    ab.ab_sync(ctx)
    torch.cuda.synchronize()
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--oracle-queries", type=int, default=131072)
    ap.add_argument("--no-also", action="store_true",
                    help="skip the secondary 16.7M-point and dense-operator measurements")
    ap.add_argument("--probe", default=None,
                    help="profiling aid: 'dense:bf16x3,tf32x3' runs one full-size dense call "
                         "per listed precision, 'c3' or 'c3:N' one clustered build, forward, "
                         "adjoint and value-and-gradient, 'bd:N' N steps of the 2-D Brownian-"
                         "dynamics loop, and exits (no timing, no JSON); 'build-paths' or "
                         "'build-paths:R' prints the median time of R builds on each "
                         "build path for the 1M, clustered 16.7M and 2-D 4M inputs")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.probe:
        probe(args.probe)
        return

    if args.impl == "reference":
        if rank != 0:
            return
        w = synth.c2()
        nq = args.oracle_queries
        pairs, secs = 0, 0.0
        for _ in range(args.warmup):
            oracle_sample(w, max(nq // 8, 1024))
        for _ in range(args.steps):
            p, dt, cores = oracle_sample(w, nq)
            pairs += p
            secs += dt
        v = pairs / secs
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "3-D uniform periodic cube, N=1048576, r=0.0197, "
                                   "Lennard-Jones sigma=0.01 eps=1: rebuild + energy + forces"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"oracle cell list over all 1048576 points + LJ energy "
                                       f"and adjoint for {nq} query particles per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    out, w = run_ours(args, rank, world)
    if rank == 0 and not args.no_also and world == 1:
        out["also"] = {"c3_clustered_16M": also_c3(), "dense_kernel_matvec": also_dense(),
                       "brownian_4M_2d": also_bd(), "paper_md_example": also_md(),
                       "kernel_solve_cg": also_solve(), "sph_3d_1M": also_sph()}
    if rank == 0:
        if world == 1:   # the host-core baseline is taken at N = 1 only
            pairs, secs, cores = oracle_sample(w, args.oracle_queries)
            out["cpu_baseline"] = {"value": pairs / secs, "unit": UNIT, "cores": cores,
                                   "kind": "oracle",
                                   "sample": f"oracle cell list over all {w.n} points + LJ energy "
                                             f"and adjoint for {args.oracle_queries} query particles"}
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
