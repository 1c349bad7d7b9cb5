"""SPH density and pressure force (Wendland C2) through the C ABI against the
oracle (GPU)."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from _helpers import dev, host, rel_err

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


def _case(dim, periodic, n, neighbours, seed):
    pos = synth.uniform_positions(n, dim, seed)
    vol = math.pi if dim == 2 else 4.0 / 3.0 * math.pi
    r = (neighbours / (vol * n)) ** (1.0 / dim)
    m = (synth.weights(n, seed + 1) * 0.5 + 1.0).astype(np.float32) / n
    A = synth.weights(n, seed + 2, "normal").astype(np.float32)
    return pos, r, m, A


@pytest.mark.parametrize("dim,periodic,n,nb", [(3, (1, 1, 1), 65536, 50), (2, (1, 0), 20000, 30),
                                               (3, (1, 1, 1), 4000, 400)])
def test_density_and_force_against_oracle(ab, ctx, dim, periodic, n, nb):
    pos, r, m, A = _case(dim, periodic, n, nb, 500 + n)
    dom = ab.Domain(dim, periodic, r)
    ab.ab_build(ctx, dom, dev(pos))
    rho = host(ab.ab_pair_sum(ctx, "sph_density", ab.OpParams(), w=dev(m)))
    wv = np.stack([m, A], 1).astype(np.float32)
    F = host(ab.ab_pair_sum(ctx, "sph_force", ab.OpParams(), w=dev(wv)))
    ab.ab_sync(ctx)
    box = oracle.Box(dim, periodic, (0,) * dim, (1,) * dim, r)
    off, idx = oracle.CellList(box, pos).neighbours()
    rho_o = oracle.pair_values("sph_density", box, pos, off, idx, w=m)
    den = oracle.abs_terms("sph_density", box, pos, off, idx, w=m)
    assert rel_err(rho, rho_o[:, 0], den[:, 0]) <= 1e-5
    F_o = oracle.pair_values("sph_force", box, pos, off, idx, w=wv)
    den_f = oracle.abs_terms("sph_force", box, pos, off, idx, w=wv)
    for k in range(dim):
        assert rel_err(F[:, k], F_o[:, k], den_f[:, k]) <= 1e-5


def test_lattice_density_and_zero_force(ab, ctx):
    M = 32
    g = np.stack(np.meshgrid(*[np.arange(M) / M] * 3, indexing="ij"), -1).reshape(-1, 3)
    pos = synth.pack4(g.astype(np.float32))
    a = 1.0 / M
    dom = ab.Domain(3, (1, 1, 1), 4.6 * a)
    ab.ab_build(ctx, dom, dev(pos))
    m = np.full(len(pos), a ** 3, np.float32)
    rho = host(ab.ab_pair_sum(ctx, "sph_density", ab.OpParams(), w=dev(m)))
    assert np.abs(rho - 1.0).max() < 1e-3
    wv = np.stack([m, np.full(len(pos), 3.0, np.float32)], 1)
    F = host(ab.ab_pair_sum(ctx, "sph_force", ab.OpParams(), w=dev(wv)))
    box = oracle.Box(3, (1, 1, 1), (0, 0, 0), (1, 1, 1), 4.6 * a)
    off, idx = oracle.CellList(box, pos).neighbours(np.arange(64))
    scale = oracle.abs_terms("sph_force", box, pos, off, idx, np.arange(64), w=wv)[:, :3].max()
    assert np.abs(F[:, :3]).max() <= 1e-5 * scale


def test_momentum_conservation(ab, ctx):
    pos, r, m, A = _case(3, (1, 1, 1), 200000, 60, 9)
    dom = ab.Domain(3, (1, 1, 1), r)
    ab.ab_build(ctx, dom, dev(pos))
    F = ab.ab_pair_sum(ctx, "sph_force", ab.OpParams(), w=dev(np.stack([m, A], 1)))
    mf = torch.from_numpy(m).to("cuda:0").double()[:, None] * F[:, :3].double()
    assert float(mf.sum(0).abs().max()) <= 1e-5 * float(mf.abs().sum())
    ab.ab_sync(ctx)


def test_sph_argument_errors(ab, ctx):
    pos, r, m, A = _case(3, (1, 1, 1), 1000, 30, 4)
    dom = ab.Domain(3, (1, 1, 1), r)
    ab.ab_build(ctx, dom, dev(pos))
    with pytest.raises(ab.AbError) as e:
        ab.ab_pair_sum(ctx, "sph_density", ab.OpParams())
    assert e.value.status == ab._abi.AB_ERR_INVALID_ARG
    wv = torch.zeros((1001, 2), dtype=torch.float32, device="cuda:0")
    with pytest.raises(ab.AbError) as e:
        ab.ab_pair_sum(ctx, "sph_force", ab.OpParams(), w=wv.view(-1)[1:2001])
    assert e.value.status == ab._abi.AB_ERR_INVALID_ARG
    ab.ab_sync(ctx)
