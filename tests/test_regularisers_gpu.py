"""GPU parity of the training-stage regularisers (Sec. 4.3): sparsity (Eq. 7)
and block opacity (Eq. 8), losses and density gradients, against the oracle
pinned in tests/test_oracle_regularisers.py.  Tolerances: loss relative
error <= 1e-4, gradient relative L2 error <= 1e-3 per tensor."""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_16457_gb300 import cow, synth, train
from gradcheck import assert_grad

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2312_16457_gb300 import build

    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _zeros(sc):
    gg = [torch.zeros(b.grid.shape, device="cuda") for b in sc.blocks]
    gp = [[torch.zeros(p.shape, device="cuda") for p in b.planes] for b in sc.blocks]
    return gg, gp


def _check_grads(gg, gp, og, op):
    for b in range(len(gg)):
        assert_grad(gg[b].cpu().numpy(), og[b], str(("grid", b)))
        for k in range(3):
            assert_grad(gp[b][k].cpu().numpy(), op[b][k], str(("plane", b, k)))
        assert torch.all(gg[b][..., 1:] == 0)


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_sparsity_matches_oracle(storage):
    sc = synth.city_scene(17, 2, 2.0, [(16, 40)])
    ctx = cow.Context(sc, storage)
    ids = list(range(4))
    pts = np.random.default_rng(2).uniform(sc.box_lo, sc.box_hi, size=(1 << 14, 3)).astype(np.float32)
    gg, gp = _zeros(sc)
    loss = ctx.sparsity_loss(torch.from_numpy(pts).cuda(), ids, 0.05, grads=(gg, gp))
    ctx.sync_check()
    osc = oracle.OracleScene(sc, values="master" if storage == "fp32" else storage)
    ol, og, op = oracle.sparsity_loss_grad(osc, ids, pts, weight=0.05)
    assert ol > 1e-3
    assert abs(float(loss.item()) - ol) <= 1e-4 * ol
    _check_grads(gg, gp, og, op)
    # loss only: same value, no gradient arrays touched
    l2 = ctx.sparsity_loss(torch.from_numpy(pts).cuda(), ids, 0.05)
    assert abs(float(l2.item()) - ol) <= 1e-4 * ol


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_opacity_matches_oracle(storage):
    sc = synth.city_scene(18, 2, 2.0, [(16, 40)])
    ctx = cow.Context(sc, storage)
    ids = list(range(4))
    o, d = synth.random_rays(4096, 8, sc.box_lo, sc.box_hi)
    gg, gp = _zeros(sc)
    loss = ctx.opacity_loss(o.cuda(), d.cuda(), ids, 0.001, grads=(gg, gp))
    ctx.sync_check()
    osc = oracle.OracleScene(sc, values="master" if storage == "fp32" else storage)
    ol, og, op = oracle.opacity_loss_grad(osc, ids, o, d, weight=0.001)
    assert ol > 1e-5
    assert abs(float(loss.item()) - ol) <= 1e-4 * ol
    _check_grads(gg, gp, og, op)
    # the same from the forward's in-block transmittances (one march a block)
    rgb, _, bt = ctx.render_rays_block_t(o.cuda(), d.cuda(), ids, synth.mlp_weights(3))
    rgb2 = ctx.render_rays(o.cuda(), d.cuda(), ids, synth.mlp_weights(3), aux=False)[0]
    assert (rgb - rgb2).abs().max().item() <= 1e-6
    assert bool(((bt == -1) | ((bt > 0) & (bt <= 1))).all()) and bool((bt == -1).any()) and bool((bt > 0).any())
    gg2, gp2 = _zeros(sc)
    loss2 = ctx.opacity_loss(o.cuda(), d.cuda(), ids, 0.001, grads=(gg2, gp2), block_T=bt)
    ctx.sync_check()
    assert abs(float(loss2.item()) - ol) <= 1e-4 * ol
    _check_grads(gg2, gp2, og, op)


def test_fitter_with_regularisers():
    """The sparsity term alone drives the mean alpha at random points down;
    with the paper's weights a fit runs and stays finite."""
    sc = synth.city_scene(4, 2, 2.0, [(24, 64)])
    fit = train.Fitter(sc, synth.mlp_weights(104), lambda_sparsity=50.0, seed=3)
    o, d = synth.random_rays(1 << 14, 4, sc.box_lo, sc.box_hi)
    o, d = o.cuda(), d.cuda()
    target = torch.zeros((o.shape[0], 3), device="cuda")
    pts = torch.from_numpy(np.random.default_rng(5).uniform(sc.box_lo, sc.box_hi, size=(1 << 14, 3))
                           .astype(np.float32)).cuda()
    before = float(fit.ctx.sparsity_loss(pts, fit.ids).item())
    for _ in range(20):
        fit.step(o, d, target)
    after = float(fit.ctx.sparsity_loss(pts, fit.ids).item())
    assert after < 0.8 * before, (before, after)
    fit2 = train.Fitter(sc, synth.mlp_weights(104), lambda_sparsity=0.05, lambda_opacity=0.001)
    tgt = cow.Context(synth.city_scene(40, 2, 2.0, [(24, 64)]), "fp32").render_rays(o, d, [0, 1, 2, 3],
                                                                                   synth.mlp_weights(140))[0]
    losses = [float(fit2.step(o, d, tgt).item()) for _ in range(15)]
    assert all(np.isfinite(losses)) and np.isfinite(float(fit2.reg_loss.item()))
    assert losses[-1] < losses[0]
