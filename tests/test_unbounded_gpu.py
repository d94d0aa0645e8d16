"""GPU parity of unbounded boundary blocks (MERF scene contraction, Eq. 16)
against the oracle pinned in tests/test_oracle_unbounded.py: per-pixel
occupied-sample counts bit-exact (the FP32 entry search, step recurrence,
contraction and occupancy decisions), colours within 1e-4 on the same stored
values; the ray form, its gradient, the batched form and the per-block MLP
form through the same blocks."""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_16457_gb300 import cow, synth
from gradcheck import assert_grad

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2312_16457_gb300 import build

    build.build()
    oracle.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("schedule", ["thread_const", "thread", "warp"])
@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_view_matches_oracle(schedule, storage):
    sc, cams, mlp = synth.workload_unbounded(R=32, P=96, width=96, height=54)
    ctx = cow.Context(sc, storage)
    ctx.set_schedule(schedule)
    order = ctx.sort_blocks(cams[0], list(range(4)))
    rgb, aux, ns = ctx.render(cams, [order], mlp, nsamp=True)
    ctx.sync_check()
    osc = oracle.OracleScene(sc, values="master" if storage == "fp32" else storage)
    r_o, a_o, n_o = oracle.render_view(osc, cams[0], order, mlp)
    ns = ns.cpu().numpy()
    assert np.array_equal(ns, n_o)
    assert np.abs(rgb.cpu().numpy() - r_o).max() <= TOL
    assert np.abs(aux.cpu().numpy() - a_o).max() <= TOL
    # the horizon: most rays leave the scene's box and end opaque in the shell
    assert (a_o[:, 7] < 0.5).mean() > 0.5 and n_o.max() > 60


def test_ray_form_and_gradient():
    sc, _, mlp = synth.workload_unbounded(R=24, P=64)
    ctx = cow.Context(sc, "fp32")
    ids = list(range(4))
    _, d = synth.random_rays(2048, 11, sc.box_lo, sc.box_hi)
    o = torch.tensor([0.25, -0.4, 0.3]).expand(2048, 3).contiguous()  # inside the scene, rays in every direction
    oc, dc = o.cuda(), d.cuda()
    rgb, aux, ns = ctx.render_rays(oc, dc, ids, mlp, nsamp=True)
    osc = oracle.OracleScene(sc)
    r_o, a_o, n_o = oracle.render_rays(osc, ids, o, d, mlp)
    assert np.array_equal(ns.cpu().numpy(), n_o)
    assert np.abs(rgb.cpu().numpy() - r_o).max() <= TOL
    g = np.random.default_rng(3).normal(size=(2048, 3)).astype(np.float32)
    gg = [torch.zeros(b.grid.shape, device="cuda") for b in sc.blocks]
    gp = [[torch.zeros(p.shape, device="cuda") for p in b.planes] for b in sc.blocks]
    gm = torch.zeros(499, device="cuda")
    ctx.render_backward(oc, dc, ids, torch.from_numpy(mlp).cuda(), aux, torch.from_numpy(g).cuda(), gg, gp, gm)
    ctx.sync_check()
    og, op, om = oracle.render_rays_grad(osc, ids, o, d, mlp, g)
    for b in range(4):
        assert_grad(gg[b].cpu().numpy(), og[b], f"grid {b}")
        for k in range(3):
            assert_grad(gp[b][k].cpu().numpy(), op[b][k], f"plane {b} {k}")
    assert_grad(gm.cpu().numpy(), om, "mlp")


def test_batched_and_block_mlp_forms():
    sc, cams, mlp = synth.workload_unbounded(R=24, P=64, width=64, height=36)
    ctx = cow.Context(sc, "bf16")
    order = ctx.sort_blocks(cams[0], list(range(4)))
    want, _, ns_w = ctx.render(cams, [order], mlp, nsamp=True)
    batch = cow.Batch(ctx, 1, 4)
    npix = batch.set_views(cams, [order])
    out = torch.empty((npix, 3), device="cuda")
    ns_b = torch.empty((npix,), dtype=torch.int32, device="cuda")
    batch.render(torch.from_numpy(mlp).cuda(), out, out_nsamp=ns_b)
    ctx.sync_check()
    assert torch.equal(ns_b, ns_w)
    assert (out - want).abs().max().item() <= 2e-6
    batch.close()
    L = 2
    w = synth.block_mlp_weights(9, 4, L)
    ctx32 = cow.Context(sc, "fp32")
    ctx32.set_block_mlps(w, L)
    rgb, _, ns = ctx32.render(cams, [order], None, nsamp=True, block_mlps=True)
    ctx32.sync_check()
    r_o, _, n_o = oracle.render_view_block_mlp(oracle.OracleScene(sc), cams[0], order, w, L)
    assert np.array_equal(ns.cpu().numpy(), n_o)
    assert np.abs(rgb.cpu().numpy() - r_o).max() <= TOL


def test_regularisers_through_unbounded_blocks():
    """Sparsity points beyond the scene's box fall in the extended regions;
    opacity rays leave through the contracted shells."""
    sc, _, _ = synth.workload_unbounded(R=24, P=64)
    ctx = cow.Context(sc, "fp32")
    ids = list(range(4))
    rng = np.random.default_rng(4)
    pts = rng.uniform([-6, -6, -3], [6, 6, 3], size=(1 << 13, 3)).astype(np.float32)
    _, d = synth.random_rays(1024, 12, sc.box_lo, sc.box_hi)
    o = torch.tensor([-0.5, 0.3, 0.2]).expand(1024, 3).contiguous()
    gg = [torch.zeros(b.grid.shape, device="cuda") for b in sc.blocks]
    gp = [[torch.zeros(p.shape, device="cuda") for p in b.planes] for b in sc.blocks]
    ls = ctx.sparsity_loss(torch.from_numpy(pts).cuda(), ids, 0.05, grads=(gg, gp))
    lo = ctx.opacity_loss(o.cuda(), d.cuda(), ids, 0.001, grads=(gg, gp))
    ctx.sync_check()
    osc = oracle.OracleScene(sc)
    ols, sg, sp = oracle.sparsity_loss_grad(osc, ids, pts, weight=0.05)
    olo, og, op = oracle.opacity_loss_grad(osc, ids, o, d, weight=0.001)
    assert ols > 1e-3 and olo > 1e-5
    assert abs(float(ls.item()) - ols) <= 1e-4 * ols
    assert abs(float(lo.item()) - olo) <= 1e-4 * olo
    for b in range(4):
        assert_grad(gg[b].cpu().numpy(), sg[b] + og[b], f"grid {b}")
        for k in range(3):
            assert_grad(gp[b][k].cpu().numpy(), sp[b][k] + op[b][k], f"plane {b} {k}")
