"""Pins of the oracle's SPH operators (paper Sec. 1: SPH among the particle
methods; Wendland C2 kernel with support r, Monaghan's symmetric pressure
force)."""
import numpy as np
import pytest

import oracle
import synth


def _lattice(m, dim):
    g = np.stack(np.meshgrid(*[np.arange(m) / m] * dim, indexing="ij"), -1).reshape(-1, dim)
    return synth.pack4(g.astype(np.float32))


@pytest.mark.parametrize("dim", [2, 3])
def test_lattice_density_tends_to_number_density(dim):
    """With m = a^dim the density of a periodic lattice (spacing a) is a
    Riemann sum of the normalised kernel: it tends to 1 as r / a grows."""
    M = 20 if dim == 3 else 40
    a = 1.0 / M
    pos = _lattice(M, dim)
    errs = []
    for ratio in (1.6, 2.6, 4.6):
        box = oracle.Box(dim, (1,) * dim, (0,) * dim, (1,) * dim, ratio * a)
        off, idx = oracle.CellList(box, pos).neighbours([0])
        rho = oracle.pair_values("sph_density", box, pos, off, idx, [0], w=np.full(len(pos), a ** dim))
        errs.append(abs(rho[0, 0] - 1.0))
    assert errs[-1] < 1e-3 and errs[0] > errs[1] > errs[-1]


def test_force_is_minus_2A_grad_density():
    """For constant A the pressure force is a_i = -2 A d(rho_i)/d(x_i):
    central differences of the density operator against the force operator."""
    n, r, A = 3000, 0.12, 0.7
    pos = synth.uniform_positions(n, 3, 77).astype(np.float64)
    m = synth.weights(n, 78) * 0.5 + 1.0
    box = oracle.Box(3, (1, 1, 1), (0, 0, 0), (1, 1, 1), r)
    q = [5, 17]
    off, idx = oracle.neighbours_brute(box, pos.astype(np.float32))
    qoff = np.concatenate([[0], np.cumsum([off[i + 1] - off[i] for i in q])])
    qidx = np.concatenate([idx[off[i]:off[i + 1]] for i in q])
    F = oracle.pair_values("sph_force", box, pos, qoff, qidx, q, w=np.stack([m, np.full(n, A)], 1))
    h = 1e-6
    for t, i in enumerate(q):
        for k in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, k] += h
            pm[i, k] -= h
            rp = oracle.pair_values64("sph_density", box, pp, qoff[t:t + 2] - qoff[t], qidx[qoff[t]:qoff[t + 1]], [i], w=m)
            rm = oracle.pair_values64("sph_density", box, pm, qoff[t:t + 2] - qoff[t], qidx[qoff[t]:qoff[t + 1]], [i], w=m)
            fd = -2.0 * A * (rp[0, 0] - rm[0, 0]) / (2 * h)
            assert abs(F[t, k] - fd) <= 1e-6 * (abs(fd) + np.abs(F[t, :3]).max())


def test_uniform_lattice_has_no_net_force_and_momentum_is_conserved():
    pos = _lattice(16, 3)
    box = oracle.Box(3, (1, 1, 1), (0, 0, 0), (1, 1, 1), 2.5 / 16)
    off, idx = oracle.CellList(box, pos).neighbours()
    w = np.stack([np.ones(len(pos)), np.full(len(pos), 2.0)], 1)
    F = oracle.pair_values("sph_force", box, pos, off, idx, w=w)
    scale = oracle.abs_terms("sph_force", box, pos, off, idx, w=w)[:, :3].max()
    assert np.abs(F[:, :3]).max() <= 1e-12 * scale
    # random masses and pressures: sum_i m_i a_i = 0 (pairwise antisymmetric)
    n = 4000
    p2 = synth.uniform_positions(n, 3, 91)
    box2 = oracle.Box(3, (1, 1, 1), (0, 0, 0), (1, 1, 1), 0.1)
    m = synth.weights(n, 92) * 0.3 + 1.0
    A = synth.weights(n, 93, "normal")
    off, idx = oracle.CellList(box2, p2).neighbours()
    F2 = oracle.pair_values("sph_force", box2, p2, off, idx, w=np.stack([m, A], 1))
    tot = (m[:, None] * F2[:, :3]).sum(axis=0)
    assert np.abs(tot).max() <= 1e-10 * np.abs(m[:, None] * F2[:, :3]).sum()


def test_kernel_vanishes_at_the_support_edge():
    pos = synth.pack4(np.array([[0.5, 0.5, 0.5], [0.5 + 0.1 * (1 - 1e-7), 0.5, 0.5]], np.float32))
    box = oracle.Box(3, (0, 0, 0), (0, 0, 0), (1, 1, 1), 0.1)
    off, idx = oracle.neighbours_brute(box, pos)
    rho = oracle.pair_values("sph_density", box, pos, off, idx, [0], w=np.array([0.0, 1.0]))
    assert 0 <= rho[0, 0] < 1e-20 * 21 / (2 * np.pi * 0.1 ** 3) + 1e-12
