"""The seeded input recipe (CPU): determinism, layout, ranges and the shape
parameters each workload is stated to have."""
import numpy as np

import synth


def test_uniform_positions_layout_and_range():
    a = synth.uniform_positions(10000, 3, 5)
    b = synth.uniform_positions(10000, 3, 5)
    assert a.dtype == np.float32 and a.shape == (10000, 4)
    assert np.array_equal(a, b)                                   # seeded
    assert not np.array_equal(a, synth.uniform_positions(10000, 3, 6))
    assert np.all(a[:, :3] >= 0) and np.all(a[:, :3] < 1)         # [0, 1), 1.0 folded
    assert np.all(a[:, 3] == 0)                                   # pad
    p2 = synth.uniform_positions(1000, 2, 5)
    assert np.all(p2[:, 2:] == 0)                                 # z and pad in 2-D
    assert abs(a[:, :3].mean() - 0.5) < 0.01                      # uniform


def test_fold_of_one():
    x = synth._to_f32_unit(np.array([0.999999999, 0.5, 1.0 - 1e-12]))
    assert x.dtype == np.float32 and np.all(x < 1) and x[0] == 0 and x[2] == 0


def test_workload_parameters():
    c1 = synth.c1()
    assert c1.n == 4096 and c1.dim == 2 and c1.radius == 0.03 and c1.periodic[:2] == (1, 1)
    assert abs(c1.params["s"] - 1e4) < 1e-6 and c1.w.min() >= -1 and c1.w.max() <= 1
    c2 = synth.c2(n=4096)
    assert c2.dim == 3 and c2.radius == 0.0197 and c2.params == {"eps": 1.0, "sigma": 0.01}
    c5 = synth.c5(n=4096)
    assert c5.dim == 2 and c5.radius == 0.002 and c5.periodic[:2] == (1, 0)
    p = synth.paper_shape(1024)
    assert abs(p.radius - (3.0 / 1024) ** 0.5) < 1e-12 and p.params["c"] == 1e-3


def test_clustered_blobs():
    w = synth.c3(n=1 << 16, n_blobs=16)
    assert w.n == 1 << 16 and w.pos.shape == (1 << 16, 4)
    assert np.all(w.pos[:, :3] >= 0) and np.all(w.pos[:, :3] < 1)
    assert abs(w.params["s"] - 1.0 / (w.radius / 3.0) ** 2) < 1e-6 * w.params["s"]
    # clustered: far more points share a small cube than under a uniform draw
    h, _ = np.histogramdd(w.pos[:, :3], bins=(32, 32, 32), range=[(0, 1)] * 3)
    assert h.max() > 20 * h.mean()


def test_dense_workload_shapes():
    d = synth.c4(m=256, n=300, nrhs=64)
    assert d.X.shape == (256, 3) and d.Y.shape == (300, 3) and d.W.shape == (300, 64)
    assert d.G.shape == (256, 64) and abs(d.s - 50.0) < 1e-9
