"""Fused LJ energy + gradient of the total energy (one walk) against the
separate forward and adjoint (bit for bit) and the oracle (GPU, C ABI)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _helpers import dev, host, oracle_box, rel_err

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


@pytest.mark.parametrize("case", ["c2", "2d", "general"])
def test_fused_equals_separate_bitwise(ab, ctx, case):
    if case == "c2":
        w = synth.c2()
        dim, periodic, r, pos = 3, w.periodic, w.radius, w.pos
    elif case == "2d":
        dim, periodic, r = 2, (1, 0), 0.02
        pos = synth.uniform_positions(200000, 2, 7)
    else:   # a periodic axis with fewer than 5 cells: the general path
        dim, periodic, r = 3, (1, 1, 1), 0.26
        pos = synth.uniform_positions(20000, 3, 8)
    prm = ab.OpParams(eps=1.0, sigma=0.01)
    dom = ab.Domain(dim, periodic, r)
    ab.ab_build(ctx, dom, dev(pos))
    n = pos.shape[0]
    e_sep = torch.empty((), dtype=torch.float64, device="cuda:0")
    E_sep = ab.ab_pair_sum(ctx, "lj", prm, energy=e_sep)
    G_sep = torch.empty((n, 4), dtype=torch.float32, device="cuda:0")
    ab.ab_pair_sum_bwd(ctx, "lj", prm, None, torch.ones(n, dtype=torch.float32, device="cuda:0"),
                       grad_pos4=G_sep)
    E, G, e = ab.ab_pair_energy_grad(ctx, "lj", prm)
    ab.ab_sync(ctx)
    assert torch.equal(E, E_sep) and torch.equal(G, G_sep) and torch.equal(e, e_sep)


def test_fused_against_oracle_sampled(ab, ctx):
    w = synth.c2()
    prm = ab.OpParams(eps=1.0, sigma=0.01)
    dom = ab.Domain(3, w.periodic, w.radius)
    ab.ab_build(ctx, dom, dev(w.pos))
    E, G, _ = ab.ab_pair_energy_grad(ctx, "lj", prm)
    q = synth.query_sample(w.n, 4096, 13)
    box = oracle_box(w)
    off, idx = oracle.CellList(box, w.pos).neighbours(q)
    Eo = oracle.pair_values("lj", box, w.pos, off, idx, q, params=w.params)
    den = oracle.abs_terms("lj", box, w.pos, off, idx, q, params=w.params)
    assert rel_err(host(E)[q], Eo[:, 0], den[:, 0]) <= 1e-5
    Go, _, _ = oracle.pair_grads("lj", box, w.pos, off, idx, np.ones(w.n), q, params=w.params)
    dg = oracle.abs_grad_terms("lj", box, w.pos, off, idx, np.ones(w.n), q, params=w.params)[0]
    for k in range(3):
        assert rel_err(host(G)[q, k], Go[:, k], dg[:, k]) <= 1e-5


def test_fused_errors(ab, ctx):
    pos = synth.uniform_positions(1000, 3, 9)
    ab.ab_build(ctx, ab.Domain(3, (1, 1, 1), 0.1), dev(pos))
    with pytest.raises(ab.AbError) as e:
        ab.ab_pair_energy_grad(ctx, "gauss", ab.OpParams(s=1.0))
    assert e.value.status == ab._abi.AB_ERR_UNSUPPORTED
    buf = torch.empty((1000, 4), dtype=torch.float32, device="cuda:0")
    with pytest.raises(ab.AbError) as e:
        ab.ab_pair_energy_grad(ctx, "lj", ab.OpParams(), E=buf.view(-1)[:1000], grad_pos4=buf)
    assert e.value.status == ab._abi.AB_ERR_ALIAS
    ab.ab_sync(ctx)


@pytest.mark.parametrize("case", ["c2", "2d", "general"])
def test_packed_layout_equals_pos4(ab, ctx, case):
    """Positions packed as dim floats per particle (ab_build_packed) and the
    packed gradient give bit for bit the pos4 results: the same cell list,
    energies, gradients and total energy (fast path, 2-D with a wall, and
    the general path of a periodic axis with fewer than 5 cells)."""
    if case == "c2":
        w = synth.c2()
        dim, periodic, r, pos = 3, w.periodic, w.radius, w.pos
    elif case == "2d":
        dim, periodic, r = 2, (1, 0), 0.02
        pos = synth.uniform_positions(200000, 2, 7)
    else:
        dim, periodic, r = 3, (1, 1, 1), 0.26
        pos = synth.uniform_positions(20000, 3, 8)
    prm = ab.OpParams(eps=1.0, sigma=0.01)
    dom = ab.Domain(dim, periodic, r)
    ab.ab_build(ctx, dom, dev(pos))
    perm4, start4 = ab.ab_cell_export(ctx)
    E4, G4, e4 = ab.ab_pair_energy_grad(ctx, "lj", prm)
    packed = dev(np.ascontiguousarray(pos[:, :dim]))
    ab.ab_build(ctx, dom, packed)
    perm, start = ab.ab_cell_export(ctx)
    E, G, e = ab.ab_pair_energy_grad_packed(ctx, "lj", prm)
    ab.ab_sync(ctx)
    assert G.shape == (pos.shape[0], dim)
    assert torch.equal(perm, perm4) and torch.equal(start, start4)
    assert torch.equal(E, E4) and torch.equal(e, e4)
    assert torch.equal(G, G4[:, :dim])


def test_packed_wrapper_and_errors(ab, ctx):
    from paper_1704_08907_gb300.autograd import lj_energy_forces
    w = synth.c2(n=1 << 16)
    dom = ab.Domain(3, w.periodic, w.radius)
    E4, F4, e4 = lj_energy_forces(ctx, dom, dev(w.pos), 1.0, 0.01)
    E, F, e = lj_energy_forces(ctx, dom, dev(np.ascontiguousarray(w.pos[:, :3])), 1.0, 0.01)
    assert F.shape == (w.n, 3) and torch.equal(F, F4[:, :3]) and torch.equal(e, e4)
    g = torch.rand(w.n, dtype=torch.float32, device="cuda:0")
    _, Fg4, _ = lj_energy_forces(ctx, dom, dev(w.pos), 1.0, 0.01, g=g)
    _, Fg, _ = lj_energy_forces(ctx, dom, dev(np.ascontiguousarray(w.pos[:, :3])), 1.0, 0.01, g=g)
    assert torch.equal(Fg, Fg4[:, :3])
    buf = torch.empty(w.n * 3, dtype=torch.float32, device="cuda:0")
    with pytest.raises(ab.AbError) as err:   # E overlapping the packed gradient
        ab.ab_pair_energy_grad_packed(ctx, "lj", ab.OpParams(eps=1.0, sigma=0.01),
                                      E=buf[: w.n], grad_pos=buf.view(w.n, 3))
    assert err.value.status == ab._abi.AB_ERR_ALIAS
    ab.ab_sync(ctx)
