"""Kernel-system solve (K(X, X) + sigma^2 I) W = B by conjugate gradients on
the library's dense operator (paper Sec. 1.1; GPU, C ABI)."""
import numpy as np
import pytest
import torch

import synth
from _helpers import dev, host
from oracle import solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ab():
    import paper_1704_08907_gb300 as ab
    return ab


@pytest.fixture(scope="module")
def ctx(ab, cuda):
    c = ab.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def system():
    n = 4096
    X = synth.uniform_positions(n, 3, 2024)
    B = np.random.default_rng(2025).standard_normal((n, 64)).astype(np.float32)
    A = solve.system_matrix(X[:, :3], 50.0, 0.1)
    return X, B, A


@pytest.mark.parametrize("prec,tol,true_tol", [("fp32", 1e-5, 5e-5), ("bf16x3", 1e-4, 5e-4),
                                               ("tf32x3", 1e-4, 5e-4)])
def test_solution_residual_against_fp64(ab, ctx, system, prec, tol, true_tol):
    """The returned W solves the FP64 system to the requested tolerance (up
    to the matvec's own error), in about as many iterations as the oracle."""
    X, B, A = system
    W, it, rr = ab.ab_kernel_solve(ctx, dev(X), dev(B), 50.0, 0.1, prec, tol, 2000)
    ab.ab_sync(ctx)
    Wh = host(W).astype(np.float64)
    true = np.linalg.norm(B - A @ Wh, axis=0) / np.linalg.norm(B, axis=0)
    assert rr <= tol and it < 2000
    assert true.max() <= true_tol
    _, it_ref, _ = solve.cg(X[:, :3], B, 50.0, 0.1, tol, 2000, A=A)
    assert abs(it - it_ref) <= max(3, 0.15 * it_ref)
    Wd = solve.direct(X[:, :3], B, 50.0, 0.1)
    assert np.linalg.norm(Wh - Wd) <= 1e3 * true.max() * np.linalg.norm(Wd)


def test_deterministic_and_edge_cases(ab, ctx, system):
    X, B, _ = system
    Xd, Bd = dev(X), dev(B)
    W1, it1, _ = ab.ab_kernel_solve(ctx, Xd, Bd, 50.0, 0.1, "bf16x3", 1e-4, 500)
    W2, it2, _ = ab.ab_kernel_solve(ctx, Xd, Bd, 50.0, 0.1, "bf16x3", 1e-4, 500)
    assert it1 == it2 and torch.equal(W1, W2)
    # a zero right-hand side stops at once with W = 0; others are unaffected
    B0 = B.copy()
    B0[:, 5] = 0.0
    W0, _, _ = ab.ab_kernel_solve(ctx, Xd, dev(B0), 50.0, 0.1, "bf16x3", 1e-4, 500)
    assert torch.all(W0[:, 5] == 0)
    # max_iter = 0 leaves W = 0
    Wz, itz, rrz = ab.ab_kernel_solve(ctx, Xd, Bd, 50.0, 0.1, "fp32", 1e-4, 0)
    assert itz == 0 and torch.all(Wz == 0) and abs(rrz - 1.0) < 1e-6
    # n = 0
    _, it0, _ = ab.ab_kernel_solve(ctx, Xd[:0], Bd[:0], 50.0, 0.1, "fp32", 1e-4, 10)
    assert it0 == 0
    # FP32 with a single column
    Wc, itc, rrc = ab.ab_kernel_solve(ctx, Xd, dev(B[:, :1].copy()), 50.0, 0.1, "fp32", 1e-5, 2000)
    assert rrc <= 1e-5 and itc > 0
    ab.ab_sync(ctx)


def test_solve_errors(ab, ctx, system):
    X, B, _ = system
    Xd, Bd = dev(X), dev(B)
    with pytest.raises(ab.AbError) as e:
        ab.ab_kernel_solve(ctx, Xd, Bd, 50.0, 0.1, "fp32", 1e-4, 10, W=Bd)
    assert e.value.status == ab._abi.AB_ERR_ALIAS
    with pytest.raises(ab.AbError) as e:
        ab.ab_kernel_solve(ctx, Xd, dev(B[:, :8].copy()), 50.0, 0.1, "bf16x3", 1e-4, 10)
    assert e.value.status == ab._abi.AB_ERR_UNSUPPORTED
    with pytest.raises(ab.AbError) as e:
        ab.ab_kernel_solve(ctx, Xd, Bd, 50.0, -1.0, "fp32", 1e-4, 10)
    assert e.value.status == ab._abi.AB_ERR_INVALID_ARG
    ab.ab_sync(ctx)
