"""Find the cut-off radius giving 64 neighbours mean for the clustered
16.7M-point workload (1024 Gaussian blobs, sd 0.01, periodic unit cube).

Calls only the oracle: bisection on r of the mean neighbour count of a fixed
65,536-point query sample against all points.  Writes c3_radius.json beside
this script; the value is copied into ``synth.C3_RADIUS``.

    python tests/golden/make_c3_radius.py
"""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "..", ".."))
import oracle  # noqa: E402
import synth  # noqa: E402


def mean_count(pos, q, r):
    box = oracle.Box(3, (1, 1, 1), radius=r)
    cl = oracle.CellList(box, pos)
    m = float(cl.counts(q).mean())
    cl.close()
    return m


def main():
    w = synth.c3(radius=0.0034)
    q = synth.query_sample(w.n, 65536, synth.BASE_SEED + 30)
    lo, hi = 0.002, 0.005
    for _ in range(22):
        mid = float(np.float32(0.5 * (lo + hi)))
        m = mean_count(w.pos, q, mid)
        print(f"r={mid:.9f} mean={m:.4f}", flush=True)
        if m < 64.0:
            lo = mid
        else:
            hi = mid
    r = float(np.float32(hi))
    out = {"radius": r, "mean_neighbours": mean_count(w.pos, q, r),
           "query_sample": 65536, "query_seed": synth.BASE_SEED + 30,
           "n": w.n, "blobs": 1024, "blob_sd": 0.01}
    with open(os.path.join(os.path.dirname(__file__), "c3_radius.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
