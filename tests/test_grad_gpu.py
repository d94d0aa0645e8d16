"""GPU parity of the differentiation form: cow_render_backward against the
oracle's FP64 analytic gradient (which tests/test_oracle_formats_lod_grad.py
pins to central finite differences), the autograd.Function path, and a short
Adam fit.  Tolerance: relative error <= 1e-3 in the L2 norm of each tensor."""
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


def _rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _gpu_grads(ctx, sc, o, d, ids, mlp, g):
    dev = "cuda"
    rgb, aux, ns = ctx.render_rays(o, d, ids, mlp, nsamp=True)
    gg = [torch.zeros(b.grid.shape, device=dev) for b in sc.blocks]
    gp = [[torch.zeros(p.shape, device=dev) for p in b.planes] for b in sc.blocks]
    gm = torch.zeros(499, device=dev)
    ctx.render_backward(o, d, ids, mlp, aux, g, gg, gp, gm)
    ctx.sync_check()
    return rgb, ns, gg, gp, gm


@pytest.mark.parametrize("storage", ["fp32", "bf16", "bf16_fp8"])
def test_backward_matches_oracle_gradient(storage):
    sc = synth.city_scene(17, 2, 2.0, [(16, 40)])
    o, d = synth.random_rays(4096, 7, sc.box_lo, sc.box_hi)
    mlp = synth.mlp_weights(8)
    g = np.random.default_rng(4).normal(size=(4096, 3)).astype(np.float32)
    ids = list(range(4))
    ctx = cow.Context(sc, storage)
    mlp_d = torch.from_numpy(mlp).cuda()
    rgb, ns, gg, gp, gm = _gpu_grads(ctx, sc, o.cuda(), d.cuda(), ids, mlp_d, torch.from_numpy(g).cuda())
    osc = oracle.OracleScene(sc, values="master" if storage == "fp32" else storage)
    og, op, om = oracle.render_rays_grad(osc, ids, o, d, mlp, g)
    _, _, n_o = oracle.render_rays(osc, ids, o, d, mlp)
    assert np.array_equal(ns.cpu().numpy(), n_o)
    assert (n_o > 0).mean() > 0.5
    for b in range(4):
        assert_grad(gg[b].cpu().numpy(), og[b], str(("grid", b)))
        for k in range(3):
            assert_grad(gp[b][k].cpu().numpy(), op[b][k], str(("plane", b, k)))
    assert_grad(gm.cpu().numpy(), om, "mlp")
    assert np.abs(om).max() > 1e-3 and max(np.abs(x).max() for x in og) > 1e-4


def test_autograd_function_matches_direct_call():
    sc = synth.city_scene(18, 2, 2.0, [(12, 24)])
    o, d = synth.random_rays(2048, 9, sc.box_lo, sc.box_hi)
    o, d = o.cuda(), d.cuda()
    ctx = cow.Context(sc, "fp32")
    ids = list(range(4))
    mlp = torch.from_numpy(synth.mlp_weights(3)).cuda().requires_grad_(True)
    params = []
    for b in sc.blocks:
        params += [b.grid.cuda().clone().requires_grad_(True)] + [p.cuda().clone().requires_grad_(True) for p in b.planes]
    wts = torch.randn(2048, 3, device="cuda")
    rgb = train.render_rays(ctx, ids, o, d, mlp, params)
    (rgb * wts).sum().backward()
    rgb2, ns, gg, gp, gm = _gpu_grads(ctx, sc, o, d, ids, mlp.detach(), wts)
    assert torch.equal(rgb, rgb2)
    assert _rel(mlp.grad.cpu().numpy(), gm.cpu().numpy()) <= 1e-6
    for b in range(4):
        assert _rel(params[4 * b].grad.cpu().numpy(), gg[b].cpu().numpy()) <= 1e-6
        for k in range(3):
            assert _rel(params[4 * b + 1 + k].grad.cpu().numpy(), gp[b][k].cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_fit_reduces_loss(storage):
    """A short fit of one scene's features and MLP to another seed's render,
    rendering from FP32 or from BF16 copies of the FP32 parameters."""
    sc = synth.city_scene(4, 2, 2.0, [(24, 64)])
    tgt_scene = synth.city_scene(40, 2, 2.0, [(24, 64)])
    o, d = synth.random_rays(1 << 16, 4, sc.box_lo, sc.box_hi)
    o, d = o.cuda(), d.cuda()
    tctx = cow.Context(tgt_scene, "fp32")
    target = tctx.render_rays(o, d, [0, 1, 2, 3], synth.mlp_weights(140), aux=False)[0]
    fit = train.Fitter(sc, synth.mlp_weights(104), storage=storage)
    losses = [float(fit.step(o, d, target).item()) for _ in range(40)]
    fit.ctx.sync_check()
    assert losses[-1] < 0.6 * losses[0], losses[::8]
    assert all(np.isfinite(losses))


def test_backward_matches_gpu_finite_differences():
    """Central differences of the GPU render itself (FP32 renders, the loss
    summed in FP64) against the analytic backward, on the entries with the
    largest gradients; h = 1e-2 keeps FP32 rounding well below the signal."""
    sc = synth.city_scene(21, 2, 2.0, [(12, 32)])
    o, d = synth.random_rays(4096, 13, sc.box_lo, sc.box_hi)
    o, d = o.cuda(), d.cuda()
    mlp = torch.from_numpy(synth.mlp_weights(5)).cuda()
    w = torch.randn(4096, 3, device="cuda", generator=torch.Generator(device="cuda").manual_seed(2))
    ctx = cow.Context(sc, "fp32")
    ids = list(range(4))
    _, _, gg, gp, gm = _gpu_grads(ctx, sc, o, d, ids, mlp, w)
    grids = [b.grid.cuda().clone() for b in sc.blocks]
    planes = [[p.cuda().clone() for p in b.planes] for b in sc.blocks]

    def loss():
        rgb = ctx.render_rays(o, d, ids, mlp, aux=False)[0]
        return float((rgb.double() * w.double()).sum())

    cands = []
    for b in range(4):
        cands.append((b, -1, gg[b]))
        cands += [(b, k, gp[b][k]) for k in range(3)]
    picks = []
    for b, k, g in cands:
        flat = g.reshape(-1)
        j = int(flat.abs().argmax())
        picks.append((b, k, j, float(flat[j])))
    h = 1e-2
    checked = 0
    for b, k, j, gval in picks:
        if abs(gval) < 0.05:
            continue
        arr = grids[b] if k < 0 else planes[b][k]
        flat = arr.view(-1)
        x0 = float(flat[j])
        vals = []
        for s in (1.0, -1.0):
            flat[j] = x0 + s * h
            ctx.update_features(b, grids[b], planes[b])
            vals.append(loss())
        flat[j] = x0
        ctx.update_features(b, grids[b], planes[b])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - gval) <= 0.03 * abs(gval) + 2e-3, (b, k, j, fd, gval)
        checked += 1
    for j in gm.abs().argsort(descending=True)[:3].tolist():  # the deferred MLP
        x0 = float(mlp[j])
        vals = []
        for s in (1.0, -1.0):
            mlp[j] = x0 + s * h
            vals.append(loss())
        mlp[j] = x0
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - float(gm[j])) <= 0.03 * abs(float(gm[j])) + 2e-3, ("mlp", j, fd, float(gm[j]))
        checked += 1
    assert checked >= 8


def test_fit_checkpoint_resumes_exactly(tmp_path):
    """A fit saved after some Adam steps and resumed in a new Fitter takes
    the same next steps as the uninterrupted one (parameters, Adam moments,
    step count and the sampler's state are all in the checkpoint)."""
    sc = synth.city_scene(4, 2, 2.0, [(12, 24)])
    tgt = synth.city_scene(40, 2, 2.0, [(12, 24)])
    o, d = synth.random_rays(1 << 13, 4, sc.box_lo, sc.box_hi)
    o, d = o.cuda(), d.cuda()
    tctx = cow.Context(tgt, "fp32")
    target = tctx.render_rays(o, d, [0, 1, 2, 3], synth.mlp_weights(140), aux=False)[0]
    a = train.Fitter(sc, synth.mlp_weights(104), lambda_sparsity=0.05)
    for _ in range(3):
        a.step(o, d, target)
    path = str(tmp_path / "fit.pt")
    a.save(path)
    la = [float(a.step(o, d, target).item()) for _ in range(3)]
    b = train.Fitter(sc, synth.mlp_weights(7), lambda_sparsity=0.05)
    b.load(path)
    lb = [float(b.step(o, d, target).item()) for _ in range(3)]
    np.testing.assert_allclose(lb, la, rtol=1e-5)
    for p, q in zip(a.params, b.params):
        assert float((p - q).abs().max()) <= 1e-5 * max(1.0, float(p.abs().max()))
    assert b.t == a.t


def test_backward_matches_fp64_gpu_central_differences():
    """Central differences of the FP64 GPU render (cow_render_rays_f64: the
    same samples, every value after them in FP64) against the FP32 backward,
    entry by entry at the differentiation form's 1e-3: the largest entries
    and random ones of every grid, plane and the deferred MLP (~80 entries)."""
    sc = synth.city_scene(21, 2, 2.0, [(12, 32)])
    o, d = synth.random_rays(4096, 13, sc.box_lo, sc.box_hi)
    o, d = o.cuda(), d.cuda()
    mlp = torch.from_numpy(synth.mlp_weights(5)).cuda()
    w = torch.randn(4096, 3, device="cuda", generator=torch.Generator(device="cuda").manual_seed(2))
    ctx = cow.Context(sc, "fp32")
    ids = list(range(4))
    _, _, gg, gp, gm = _gpu_grads(ctx, sc, o, d, ids, mlp, w)
    g64 = [b.grid.double().cuda().contiguous() for b in sc.blocks]
    p64 = [[p.double().cuda().contiguous() for p in b.planes] for b in sc.blocks]
    m64 = mlp.double().clone()
    w64 = w.double()

    def loss():
        rgb, _ = ctx.render_rays_f64(o, d, ids, m64, g64, p64)
        return float((rgb * w64).sum())

    # the FP64 render and the FP32 render agree (same samples)
    rgb32 = ctx.render_rays(o, d, ids, mlp, aux=False)[0]
    rgb64, _ = ctx.render_rays_f64(o, d, ids, m64, g64, p64)
    assert float((rgb64 - rgb32.double()).abs().max()) <= 1e-5
    rng = np.random.default_rng(9)
    targets = []
    for b in range(4):
        targets.append((g64[b], gg[b]))
        targets += [(p64[b][k], gp[b][k]) for k in range(3)]
    targets.append((m64, gm))
    checked = skipped = 0
    l0 = loss()
    for x64, g in targets:
        flat_g = g.reshape(-1)
        scale = float(flat_g.abs().max())
        big = torch.nonzero(flat_g.abs() >= 0.05 * scale).reshape(-1).cpu().numpy()
        picks = list(flat_g.abs().argsort(descending=True)[:2].tolist())
        if len(big):
            picks += list(rng.choice(big, size=min(3, len(big)), replace=False))
        xf = x64.view(-1)

        def central(j, h):
            x0 = float(xf[j])
            xf[j] = x0 + h
            lp = loss()
            xf[j] = x0 - h
            lm = loss()
            xf[j] = x0
            return (lp - lm) / (2 * h)

        for j in dict.fromkeys(int(v) for v in picks):
            # small steps (the FP64 loss rounds at ~1e-14 of its size), taken
            # twice: where the two disagree a ReLU of the deferred MLP changes
            # sign inside the step for some ray, so the difference quotient is
            # not the derivative there and the entry is skipped
            h = 1e-6 * max(1.0, abs(float(xf[j])))
            fd, fd2 = central(j, h), central(j, 2 * h)
            if abs(fd - fd2) > 1e-5 * max(abs(fd), 1e-2 * scale) + 1e-13 * abs(l0) / h:
                skipped += 1
                continue
            gv = float(flat_g[j])
            bound = 1e-3 * abs(fd) if abs(fd) >= 1e-2 * scale else 1e-3 * scale
            assert abs(fd - gv) <= bound, (j, fd, gv, scale)
            checked += 1
    assert checked >= 60 and skipped <= 4, (checked, skipped)


def test_coherent_ray_order_keeps_results():
    """The coherent processing order of ray batches (the default for 8192
    rays or more) writes every ray's forward outputs and per-block partials
    bit for bit as the given order does, and the same gradients up to the
    order of their FP32 reductions (global and per-block MLP forms)."""
    sc = synth.city_scene(21, 2, 2.0, [(12, 32)])
    n = 20000
    o, d = synth.random_rays(n, 13, sc.box_lo, sc.box_hi)
    o, d = o.cuda(), d.cuda()
    mlp = torch.from_numpy(synth.mlp_weights(5)).cuda()
    g = torch.randn(n, 3, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    ctx = cow.Context(sc, "fp32")
    ids = list(range(4))
    res = {}
    for mode in ("given", "coherent"):
        ctx.set_ray_order(mode)
        rgb, ns, gg, gp, gm = _gpu_grads(ctx, sc, o, d, ids, mlp, g)
        part = ctx.render_partials(o, d, ids)
        ctx.sync_check()
        res[mode] = (rgb, ns, gg, gp, gm, part)
    a, b = res["given"], res["coherent"]
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) and torch.equal(a[5], b[5])
    for x, y in [*zip(a[2], b[2]), *[(p, q) for pa, pb in zip(a[3], b[3]) for p, q in zip(pa, pb)], (a[4], b[4])]:
        assert float((x - y).abs().max()) <= 1e-5 * float(x.abs().max()) + 1e-12
    # per-block MLP form
    nb, L = len(sc.blocks), 2
    ctx.set_block_mlps(synth.block_mlp_weights(13, nb, L), L)
    res = {}
    for mode in ("given", "coherent"):
        ctx.set_ray_order(mode)
        rgb = ctx.render_rays(o, d, ids, None, aux=False, block_mlps=True)[0]
        gg = [torch.zeros(bk.grid.shape, device="cuda") for bk in sc.blocks]
        gp = [[torch.zeros(p.shape, device="cuda") for p in bk.planes] for bk in sc.blocks]
        gw = torch.zeros((nb, synth.block_mlp_nparam(L)), device="cuda")
        ctx.render_backward_block_mlps(o, d, ids, g, gg, gp, gw)
        ctx.sync_check()
        res[mode] = (rgb, gg, gw)
    a, b = res["given"], res["coherent"]
    assert torch.equal(a[0], b[0])
    for x, y in [*zip(a[1], b[1]), (a[2], b[2])]:
        assert float((x - y).abs().max()) <= 1e-5 * float(x.abs().max()) + 1e-12
    ctx.close()
