"""GPU parity of the per-block deferred-MLP form (Sec. 4.1: one MLP per block
and LOD level; Sec. 4.2, Eq. 5 with Eq. 3 per block) with a multi-frequency
PE(d), against the oracle pinned in tests/test_oracle_block_mlp.py.

Tolerances as for the global form: plain FP32 math max |dRGB| <= 1e-4 against
the oracle on the same stored values, occupied-sample counts bit-exact;
BF16 storage PSNR >= 45 dB and max |dRGB| <= 1e-2 against the FP32 master."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2312_16457_gb300 import cow, synth, train
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


def _render(ctx, cams, ids, **kw):
    rgb, aux, ns = ctx.render(cams, ids, None, nsamp=True, block_mlps=True, **kw)
    ctx.sync_check()
    return rgb.cpu().numpy(), aux.cpu().numpy(), ns.cpu().numpy()


def _psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return math.inf if mse == 0 else 10 * math.log10(1.0 / mse)


@pytest.mark.parametrize("schedule", ["thread", "thread_const", "warp"])
@pytest.mark.parametrize("n_freq", [0, 4])
def test_fp16_storage_matches_oracle(schedule, n_freq):
    sc, cams, _ = synth.workload_city_4x4(R=48, P=160, width=200, height=120)
    n = len(sc.blocks)
    w = synth.block_mlp_weights(11, n, n_freq, spread=0.3)
    ctx = cow.Context(sc, "fp16")
    ctx.set_schedule(schedule)
    ctx.set_block_mlps(w, n_freq)
    order = ctx.sort_blocks(cams[0], list(range(n)))
    rgb, aux, ns = _render(ctx, cams, [order])
    osc = oracle.OracleScene(sc, values="fp16")
    r_o, a_o, n_o = oracle.render_view_block_mlp(osc, cams[0], order, w, n_freq)
    assert np.array_equal(ns, n_o)
    assert (n_o > 0).mean() > 0.5
    assert np.abs(rgb - r_o).max() <= TOL
    assert np.abs(aux - a_o).max() <= TOL
    # early termination at 1e-5 stays within the tolerance
    rgb_e, _, ns_e = _render(ctx, cams, [order], ert_eps=1e-5)
    assert np.abs(rgb_e - r_o).max() <= TOL
    assert ns_e.sum() < ns.sum()


def test_bf16_storage_lod_city():
    """LOD city (3 levels, every block its own MLP), BF16 storage, against the
    oracle on the FP32 master."""
    sc, cams, _ = synth.workload_city_lod(res=((48, 160), (24, 80), (12, 40)), width=192, height=108)
    n = len(sc.blocks)
    L = 4
    w = synth.block_mlp_weights(12, n, L)
    ctx = cow.Context(sc, "bf16")
    ctx.set_block_mlps(torch.from_numpy(w).cuda(), L)  # device source
    ids = ctx.select_lod(cams[0], sc.lod_thresh)
    assert len({sc.blocks[i].level for i in ids}) >= 2
    rgb, aux, ns = _render(ctx, cams, [ids])
    osc = oracle.OracleScene(sc)
    r_o, _, n_o = oracle.render_view_block_mlp(osc, cams[0], ids, w, L)
    assert (n_o > 0).mean() > 0.35
    assert _psnr(rgb, r_o) >= 45.0
    assert np.abs(rgb - r_o).max() <= 1e-2


def test_multiview_equals_single_views():
    sc, _, _ = synth.workload_city_4x4(R=24, P=48)
    n = len(sc.blocks)
    ctx = cow.Context(sc, "bf16")
    ctx.set_block_mlps(synth.block_mlp_weights(13, n, 2), 2)
    cams = [synth.camera((0.3, -7.0, 6.0), (0.0, 0.0, -1.0), 33, 17, 60.0),
            synth.camera((5.0, 1.0, 3.0), (-1.0, 0.5, -1.0), 64, 64, 45.0)]
    ids = [ctx.sort_blocks(c, list(range(n))) for c in cams]
    rgb, aux, ns = _render(ctx, cams, ids)
    off = 0
    for c, i in zip(cams, ids):
        r1, a1, n1 = _render(ctx, [c], [i])
        k = c.width * c.height
        assert np.array_equal(ns[off:off + k], n1)
        assert np.abs(rgb[off:off + k] - r1).max() <= 1e-6
        off += k


def test_argument_errors():
    sc, cams, mlp = synth.workload_single_block(R=16, P=32, width=8, height=8)
    ctx = cow.Context(sc, "fp32")
    with pytest.raises(cow.CowError):
        ctx.render(cams, [[0]], None, block_mlps=True)  # none set
    with pytest.raises(cow.CowError):
        ctx.set_block_mlps(synth.block_mlp_weights(1, 2, 0), 0)  # 2 MLPs for 1 block
    with pytest.raises(cow.CowError):
        ctx.set_block_mlps(synth.block_mlp_weights(1, 1, 9), 9)  # n_freq > 8
    ctx.set_block_mlps(synth.block_mlp_weights(1, 1, 1), 1)
    with pytest.raises(cow.CowError):
        ctx.render(cams, [[0]], None, block_mlps=True, mlp_bf16=True)
    rgb, _, _ = _render(ctx, cams, [[0]])
    assert np.isfinite(rgb).all()
    ctx.set_block_mlps(None, 0)
    with pytest.raises(cow.CowError):
        ctx.render(cams, [[0]], None, block_mlps=True)
    # the global form is unaffected
    ctx.render(cams, [[0]], mlp)
    ctx.sync_check()


def test_identical_block_mlps_seam_only_where_blocks_meet():
    """The library's per-block form with the same MLP in every block against
    its global form: equal colours on rays whose occupied samples lie in one
    block, different colours on rays with samples in two or more blocks (the
    per-block form's seam for view-dependent colour); the blended C_d, F and
    T agree everywhere."""
    sc = synth.city_scene(6, 2, 2.0, [(24, 64)])
    n = len(sc.blocks)
    mlp = synth.mlp_weights(106)
    ctx = cow.Context(sc, "fp32")
    ctx.set_block_mlps(np.repeat(mlp[None, :], n, axis=0), 0)
    cam = synth.camera((-0.6, -4.0, 3.0), (0.2, 0.3, -0.5), 80, 60, 70.0)
    order = ctx.sort_blocks(cam, list(range(n)))
    r_b, a_b, n_b = _render(ctx, [cam], [order])
    rg, ag, ng = ctx.render([cam], [order], torch.from_numpy(mlp).cuda(), nsamp=True)
    ctx.sync_check()
    r_g, a_g, n_g = rg.cpu().numpy(), ag.cpu().numpy(), ng.cpu().numpy()
    assert np.array_equal(n_b, n_g)
    assert np.abs(a_b - a_g).max() <= 1e-5
    blocks_hit = np.zeros_like(n_b)
    for k in order:
        _, _, n_k = _render(ctx, [cam], [[k]])
        blocks_hit += n_k > 0
    one, many = blocks_hit == 1, blocks_hit >= 2
    assert one.mean() > 0.15 and many.mean() > 0.05
    assert np.abs(r_b[one] - r_g[one]).max() <= 1e-5
    assert np.abs(r_b[many] - r_g[many]).max() > 1e-2


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_ray_form_matches_oracle(storage):
    """Independent rays with per-block MLPs (Eq. 5, each ray sorting the
    blocks from its own origin) against the oracle on the same values."""
    sc = synth.city_scene(6, 2, 2.0, [(24, 64)])
    n = len(sc.blocks)
    L = 4
    w = synth.block_mlp_weights(12, n, L, spread=0.3)
    ctx = cow.Context(sc, storage)
    ctx.set_block_mlps(w, L)
    o, d = synth.random_rays(4096, 9, sc.box_lo, sc.box_hi, device="cuda")
    ids = list(range(n))
    rgb, aux, ns = ctx.render_rays(o, d, ids, None, nsamp=True, block_mlps=True)
    rgb_e = ctx.render_rays(o, d, ids, None, ert_eps=1e-5, block_mlps=True)[0]
    ctx.sync_check()
    osc = oracle.OracleScene(sc, values="master" if storage == "fp32" else storage)
    r_o, a_o, n_o = oracle.render_rays_block_mlp(osc, ids, o.cpu(), d.cpu(), w, L)
    assert np.array_equal(ns.cpu().numpy(), n_o)
    assert (n_o > 0).mean() > 0.5
    assert np.abs(rgb.cpu().numpy() - r_o).max() <= TOL
    assert np.abs(aux.cpu().numpy() - a_o).max() <= TOL
    assert np.abs(rgb_e.cpu().numpy() - r_o).max() <= TOL
    # the global form on the same rays differs (the blocks' MLPs are not the global one)
    g = ctx.render_rays(o, d, ids, torch.from_numpy(synth.mlp_weights(1)).cuda())[0]
    assert float((g - rgb).abs().max()) > 1e-2


def test_ray_form_argument_errors():
    sc = synth.city_scene(6, 2, 2.0, [(12, 32)])
    ctx = cow.Context(sc, "fp32")
    o, d = synth.random_rays(64, 9, sc.box_lo, sc.box_hi, device="cuda")
    with pytest.raises(cow.CowError):  # no per-block MLPs set
        ctx.render_rays(o, d, [0, 1], None, block_mlps=True)
    ctx.set_block_mlps(synth.block_mlp_weights(1, len(sc.blocks), 0), 0)
    with pytest.raises(cow.CowError):  # the per-block MLPs run in FP32
        ctx.render_rays(o, d, [0, 1], None, block_mlps=True, mlp_bf16=True)
    with pytest.raises(cow.CowError):  # the global form needs its MLP
        ctx.render_rays(o, d, [0, 1], None)
    rgb = ctx.render_rays(o, d, [0, 1], None, block_mlps=True)[0]
    ctx.sync_check()
    assert torch.isfinite(rgb).all()


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_ray_form_backward_matches_oracle_gradient(storage):
    """cow_render_backward_block_mlps against the oracle's FP64 adjoint of the
    per-block form (pinned by central differences): relative L2 error <= 1e-3
    for every grid, plane and per-block MLP."""
    sc = synth.city_scene(17, 2, 2.0, [(16, 40)])
    n = len(sc.blocks)
    L = 2
    w = synth.block_mlp_weights(9, n, L, spread=0.3)
    o, d = synth.random_rays(4096, 7, sc.box_lo, sc.box_hi)
    g = np.random.default_rng(4).normal(size=(4096, 3)).astype(np.float32)
    ids = list(range(n))
    ctx = cow.Context(sc, storage)
    ctx.set_block_mlps(w, L)
    gg = [torch.zeros(b.grid.shape, device="cuda") for b in sc.blocks]
    gp = [[torch.zeros(p.shape, device="cuda") for p in b.planes] for b in sc.blocks]
    gm = torch.zeros(w.shape, device="cuda")
    ctx.render_backward_block_mlps(o.cuda(), d.cuda(), ids, torch.from_numpy(g).cuda(), gg, gp, gm)
    ctx.sync_check()
    osc = oracle.OracleScene(sc, values="master" if storage == "fp32" else storage)
    og, op, om = oracle.render_rays_block_mlp_grad(osc, ids, o, d, w, L, g)
    for b in range(n):
        assert_grad(gg[b].cpu().numpy(), og[b], str(("grid", b)))
        for k in range(3):
            assert_grad(gp[b][k].cpu().numpy(), op[b][k], str(("plane", b, k)))
        assert_grad(gm[b].cpu().numpy(), om[b], str(("mlp", b)))
    assert max(np.abs(x).max() for x in og) > 1e-4 and np.abs(om).max() > 1e-3
    # a second call accumulates
    ctx.render_backward_block_mlps(o.cuda(), d.cuda(), ids, torch.from_numpy(g).cuda(), gg, gp, gm)
    ctx.sync_check()
    assert_grad(gm.cpu().numpy(), 2 * om, "mlp")


def test_fit_with_block_mlps_reduces_loss():
    """A short fit of one scene's features and per-block MLPs (Eq. 5 form)
    to another seed's render."""
    sc = synth.city_scene(4, 2, 2.0, [(24, 64)])
    tgt_scene = synth.city_scene(40, 2, 2.0, [(24, 64)])
    o, d = synth.random_rays(1 << 16, 4, sc.box_lo, sc.box_hi)
    o, d = o.cuda(), d.cuda()
    tctx = cow.Context(tgt_scene, "fp32")
    target = tctx.render_rays(o, d, [0, 1, 2, 3], synth.mlp_weights(140), aux=False)[0]
    w = synth.block_mlp_weights(104, len(sc.blocks), 2)
    fit = train.Fitter(sc, None, block_mlps=w, n_freq=2)
    losses = [float(fit.step(o, d, target).item()) for _ in range(40)]
    fit.ctx.sync_check()
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.85 * losses[0], losses[::8]
    # the fitted per-block MLPs are the context's
    assert not np.allclose(fit.block_mlps.cpu().numpy(), w)


def test_backward_from_forward_state():
    """The forward that keeps every (ray, block) state renders the same
    pixels as the per-block MLP forward, and the backward from that state
    gives the gradients of the two-march backward (FP32 reduction order
    aside)."""
    sc = synth.city_scene(23, 2, 2.0, [(12, 32)])
    n, L = 20000, 2
    o, d = synth.random_rays(n, 5, sc.box_lo, sc.box_hi)
    o, d = o.cuda(), d.cuda()
    nb = len(sc.blocks)
    ids = list(range(nb))
    ctx = cow.Context(sc, "fp32")
    ctx.set_block_mlps(synth.block_mlp_weights(14, nb, L), L)
    g = torch.randn(n, 3, device="cuda", generator=torch.Generator(device="cuda").manual_seed(6))
    ref = ctx.render_rays(o, d, ids, None, aux=False, block_mlps=True)[0]
    rgb, state = ctx.render_rays_block_state(o, d, ids)
    ctx.sync_check()
    assert torch.equal(rgb, ref)
    T = state[..., 7]
    assert bool(((T == -1.0) | ((T >= 0.0) & (T <= 1.0))).all()) and bool((T >= 0.0).any())
    out = []
    for use_state in (False, True):
        gg = [torch.zeros(b.grid.shape, device="cuda") for b in sc.blocks]
        gp = [[torch.zeros(p.shape, device="cuda") for p in b.planes] for b in sc.blocks]
        gw = torch.zeros((nb, synth.block_mlp_nparam(L)), device="cuda")
        if use_state:
            ctx.render_backward_block_mlps_state(o, d, ids, state, g, gg, gp, gw)
        else:
            ctx.render_backward_block_mlps(o, d, ids, g, gg, gp, gw)
        ctx.sync_check()
        out.append((gg, gp, gw))
    a, b = out
    pairs = [*zip(a[0], b[0]), *[(x, y) for pa, pb in zip(a[1], b[1]) for x, y in zip(pa, pb)], (a[2], b[2])]
    for x, y in pairs:
        assert float((x - y).abs().max()) <= 1e-5 * float(x.abs().max()) + 1e-12
    assert float(a[2].abs().max()) > 0.0
    ctx.close()
