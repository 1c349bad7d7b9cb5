"""Pins of the oracle's kernel-system solve (paper Sec. 1.1)."""
import numpy as np

from oracle import dense, solve


def _pts(n, seed):
    return np.random.default_rng(seed).uniform(0, 1, (n, 3))


def test_cg_matches_direct_solve():
    X = _pts(300, 1)
    B = np.random.default_rng(2).standard_normal((300, 5))
    s, sigma2 = 50.0, 1e-2
    Wd = solve.direct(X, B, s, sigma2)
    Wc, it, rr = solve.cg(X, B, s, sigma2, 1e-12, 2000)
    assert rr.max() <= 1e-12 and it < 2000
    assert np.abs(Wc - Wd).max() <= 1e-8 * np.abs(Wd).max()


def test_interpolation_is_exact_at_the_nodes():
    """sigma2 = 0: the interpolant sum_j w_j K(x, x_j) reproduces y at x_i."""
    g = np.stack(np.meshgrid(*[np.arange(5) / 5.0] * 3, indexing="ij"), -1).reshape(-1, 3)
    y = np.sin(3 * g[:, :1]) + g[:, 1:2] * g[:, 2:3]
    w = solve.direct(g, y, 50.0, 0.0)
    assert np.abs(dense.matvec(g, g, w, 50.0) - y).max() < 1e-10


def test_cg_terminates_within_n_steps():
    """In exact arithmetic CG solves an SPD system in at most n iterations.
    For this 12 x 12 system (condition ~9.4) the generic rate bound would
    still allow a residual ~3e-4 after 12 steps; CG reaches FP64 rounding."""
    X = _pts(12, 3)
    B = np.random.default_rng(4).standard_normal((12, 3))
    _, it, rr = solve.cg(X, B, 5.0, 0.5, 1e-10, 100)
    assert it <= 12 and rr.max() <= 1e-10


def test_recurrence_residual_tracks_the_true_residual():
    X = _pts(400, 5)
    B = np.random.default_rng(6).standard_normal((400, 4))
    A = solve.system_matrix(X, 50.0, 0.1)
    W, it, rr = solve.cg(X, B, 50.0, 0.1, 1e-6, 1000, A=A)
    true = np.linalg.norm(B - A @ W, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(rr <= 1e-6) and np.all(true <= 2e-6)
