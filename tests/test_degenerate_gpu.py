"""Degenerate inputs of the ray-batch, regulariser, per-block MLP, unbounded
and residency calls: empty batches do nothing and succeed, a view with no
blocks renders the empty-feature colour, a budget equal to a call's need
suffices."""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_16457_gb300 import cow, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2312_16457_gb300 import build

    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def test_empty_batches():
    sc = synth.city_scene(3, 2, 2.0, [(8, 16)])
    ctx = cow.Context(sc, "fp32")
    mlp = torch.from_numpy(synth.mlp_weights(1)).cuda()
    z = torch.zeros((0, 3), device="cuda")
    rgb, aux, ns = ctx.render_rays(z, z, [0, 1, 2, 3], mlp, nsamp=True)
    assert rgb.shape == (0, 3) and ns.shape == (0,)
    gg = [torch.zeros(b.grid.shape, device="cuda") for b in sc.blocks]
    gp = [[torch.zeros(p.shape, device="cuda") for p in b.planes] for b in sc.blocks]
    gm = torch.zeros(499, device="cuda")
    ctx.render_backward(z, z, [0, 1, 2, 3], mlp, torch.zeros((0, 8), device="cuda"), z, gg, gp, gm)
    ls = ctx.sparsity_loss(z, [0, 1, 2, 3], 1.0, grads=(gg, gp))
    lo = ctx.opacity_loss(z, z, [0, 1, 2, 3], 1.0, grads=(gg, gp))
    ctx.sync_check()
    assert float(ls.item()) == 0.0 and float(lo.item()) == 0.0
    assert float(gm.abs().sum()) == 0.0 and all(float(g.abs().sum()) == 0.0 for g in gg)


def test_view_without_blocks_per_block_and_unbounded():
    """No blocks: the per-block form renders 0 (no block takes part), the
    global form sigmoid(MLP(0, 0, d)); the same through unbounded blocks."""
    sc, cams, mlp = synth.workload_unbounded(R=12, P=24, width=17, height=9)
    ctx = cow.Context(sc, "fp32")
    ctx.set_block_mlps(synth.block_mlp_weights(2, 4, 1), 1)
    rgb, aux, ns = ctx.render(cams, [[]], None, nsamp=True, block_mlps=True)
    assert torch.all(rgb == 0) and torch.all(ns == 0) and torch.all(aux[:, 7] == 1)
    rgb_g, _, _ = ctx.render(cams, [[]], mlp)
    r_o, _, _ = oracle.render_view(oracle.OracleScene(sc), cams[0], [], mlp)
    assert np.abs(rgb_g.cpu().numpy() - r_o).max() <= 1e-4
    ctx.sync_check()


def test_budget_equal_to_the_need():
    sc = synth.city_scene(3, 2, 2.0, [(8, 16)])
    ctx = cow.Context(sc, "bf16")
    cam = synth.camera((0.0, -5.0, 3.0), (0.0, 0.0, 0.0), 24, 16, 60.0)
    ids = list(range(4))
    want = ctx.render([cam], [ids], synth.mlp_weights(1))[0]
    ctx.set_residency(sum(ctx.block_bytes(i) for i in ids))
    got = ctx.render([cam], [ids], synth.mlp_weights(1))[0]
    ctx.sync_check()
    assert torch.equal(got, want)
    assert ctx.residency()["resident_blocks"] == 4
