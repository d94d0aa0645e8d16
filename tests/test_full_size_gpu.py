"""Parity at full size, in the launch configurations the benchmark times.

The oracle cannot render whole frames of these workloads within a test's
time, so each test renders the full workload on the GPU and checks sampled
outputs that the oracle computes one by one:

* the 8x8-block, 3-LOD city (256^3 / 1024^2 at LOD 1) at 1920x1080, per
  storage format, through the default view schedule;
* the 16x16-block, 3-LOD city, 64 views of mixed size, through one
  persistent, autotuned, graph-replayed batch launch;
* the 2x2-block FP32 fit scene with 2^20 random rays: the forward on sampled
  rays, and the backward of one full 2^20-ray launch whose upstream gradient
  is non-zero on the sampled rays only, against the oracle's FP64 gradient
  of those rays.

Tolerances: FP32 max |dRGB| <= 1e-4 against the oracle; BF16 and
BF16-grid / FP8-plane storage PSNR >= 45 dB and max |dRGB| <= 1e-2 against
the oracle on the FP32 master, <= 1e-4 against the oracle on the same stored
values; gradient relative error <= 1e-3; sample counts bit-exact.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2312_16457_gb300 import cow, synth
from gradcheck import assert_grad

pytestmark = pytest.mark.gpu

TOL = 1e-4
ERT = 1e-5  # the benchmark's early-termination threshold


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2312_16457_gb300 import build

    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return math.inf if mse == 0 else 10 * math.log10(1.0 / mse)


def _host_sub_scene(sc, ids):
    """The selected blocks, copied to the host and re-indexed in list order."""
    blocks = [synth.Block(sc.blocks[int(i)].lo, sc.blocks[int(i)].hi, sc.blocks[int(i)].R, sc.blocks[int(i)].P, 1, -1,
                          sc.blocks[int(i)].grid.to("cpu"), [p.to("cpu") for p in sc.blocks[int(i)].planes])
              for i in ids]
    return synth.Scene(blocks, sc.box_lo, sc.box_hi, [], sc.occ_cell, sc.occ_thresh)


def _pixels(W, H, n, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([rng.integers(0, W * H, n), [0, W - 1, W * (H - 1), W * H - 1,
                                                                (H // 2) * W + W // 2]]))


# ---------------------------------------------------------------------------
# the 1080p LOD city (the frame-rate benchmark)


@pytest.fixture(scope="module")
def city_lod():
    sc, cams, mlp = synth.workload_city_lod(device="cuda")
    cam = cams[0]
    ctx = cow.Context(sc, "fp32")
    ids = ctx.select_lod(cam, sc.lod_thresh)
    ctx.close()
    host = _host_sub_scene(sc, ids)
    pix = _pixels(cam.width, cam.height, 400, 11)
    master = oracle.OracleScene(host)
    order = list(range(len(ids)))
    r_m, a_m, n_m = oracle.render_view(master, cam, order, mlp, pixels=pix)
    yield {"sc": sc, "cam": cam, "mlp": mlp, "ids": ids, "host": host, "pix": pix, "order": order,
           "oracle_master": (r_m, a_m, n_m)}
    del sc
    torch.cuda.empty_cache()


@pytest.mark.parametrize("storage", ["fp32", "bf16", "bf16_fp8", "fp8_bf16d", "fp8"])
def test_city_lod_1080p_sampled(city_lod, storage):
    c = city_lod
    cam, ids, pix, mlp = c["cam"], c["ids"], c["pix"], c["mlp"]
    assert len(ids) == 22  # 16 LOD-1 + 4 LOD-2 + 2 LOD-3 blocks
    ctx = cow.Context(c["sc"], storage)
    assert ctx.schedule == "thread_const"
    mlp_d = torch.from_numpy(mlp).cuda()
    # the benchmark's launch: early termination on
    rgb = ctx.render([cam], [ids], mlp_d, ert_eps=ERT, aux=False)[0]
    # the definition: no early termination, sample counts kept
    rgb0, aux0, ns0 = ctx.render([cam], [ids], mlp_d, nsamp=True)
    ctx.sync_check()
    rgb = rgb.cpu().numpy()[pix]
    rgb0, aux0, ns0 = rgb0.cpu().numpy()[pix], aux0.cpu().numpy()[pix], ns0.cpu().numpy()[pix]
    ctx.close()
    r_m, a_m, n_m = c["oracle_master"]
    assert (n_m > 0).mean() > 0.3  # the upper part of the frame is sky
    assert np.array_equal(ns0, n_m)  # occupancy comes from the FP32 master in every format
    if storage == "fp32":
        assert np.abs(rgb0 - r_m).max() <= TOL
        assert np.abs(aux0 - a_m).max() <= TOL
        assert np.abs(rgb - r_m).max() <= TOL
        return
    # the same stored values in the oracle
    stored = oracle.OracleScene(c["host"], values=storage)
    r_s, a_s, n_s = oracle.render_view(stored, cam, c["order"], mlp, pixels=pix)
    del stored
    assert np.array_equal(ns0, n_s)
    assert np.abs(rgb0 - r_s).max() <= TOL
    assert np.abs(aux0[:, :7] - a_s[:, :7]).max() <= TOL
    assert np.abs(rgb - r_s).max() <= TOL
    # the format against the FP32 master (pure per-channel E4M3 is checked on
    # its stored values and for PSNR only: it does not meet the 1e-2 bound)
    assert psnr(rgb, r_m) >= 45.0
    if storage != "fp8":
        assert np.abs(rgb - r_m).max() <= 1e-2


def test_city_lod_1080p_bricks_whole_frame():
    """The 1080p LOD city baked with the sparse generator setting, brick-sparse
    BF16 grids against dense BF16 grids in the benchmark's launch: the whole
    frame bit for bit, with fewer device bytes."""
    sc, cams, mlp = synth.workload_city_lod(device="cuda", sparse=True)
    cam = cams[0]
    dense = cow.Context(sc, "bf16")
    sparse = cow.Context(sc, "bf16", bricks=True)
    ids = dense.select_lod(cam, sc.lod_thresh)
    nb = len(sc.blocks)
    del sc
    mlp_d = torch.from_numpy(mlp).cuda()
    for ert in (1e-5, 0.0):
        a = dense.render([cam], [ids], mlp_d, ert_eps=ert, nsamp=True)
        b = sparse.render([cam], [ids], mlp_d, ert_eps=ert, nsamp=True)
        dense.sync_check()
        sparse.sync_check()
        for x, y in zip(a, b):
            assert torch.equal(x, y), ert
    assert float((a[2] > 0).float().mean()) > 0.3
    bd = sum(dense.block_bytes(i) for i in range(nb))
    bs = sum(sparse.block_bytes(i) for i in range(nb))
    print(f"sparse city: dense {bd / 1e9:.2f} GB, brick-sparse {bs / 1e9:.2f} GB")
    assert bs < 0.7 * bd
    dense.close()
    sparse.close()


# ---------------------------------------------------------------------------
# 64 views in one persistent launch (the batched benchmark)


def test_batch_64_views_sampled():
    sc, cams, mlp = synth.workload_batch(device="cuda")
    ctx = cow.Context(sc, "bf16")
    ids = [ctx.select_lod(c, sc.lod_thresh) for c in cams]
    mlp_d = torch.from_numpy(mlp).cuda()
    b = cow.Batch(ctx, len(cams), sum(len(i) for i in ids))
    npix = b.set_views(cams, ids)
    assert npix == sum(c.width * c.height for c in cams)
    out = torch.empty((npix, 3), device="cuda")
    b.tune(mlp_d, out, ert_eps=ERT)
    out.zero_()
    b.render(mlp_d, out, ert_eps=ERT, graph=True)
    ctx.sync_check()
    rgb = out.cpu().numpy()
    b.close()
    ctx.close()
    offs = np.concatenate([[0], np.cumsum([c.width * c.height for c in cams])])
    # one view of each size, plus the view with the most blocks
    picks = []
    for size in sorted({(c.width, c.height) for c in cams}):
        picks.append(next(v for v, c in enumerate(cams) if (c.width, c.height) == size))
    picks.append(int(np.argmax([len(i) for i in ids])))
    for v in sorted(set(picks)):
        cam = cams[v]
        host = _host_sub_scene(sc, ids[v])
        pix = _pixels(cam.width, cam.height, 96, 100 + v)
        order = list(range(len(ids[v])))
        got = rgb[offs[v] + pix]
        r_s, _, n_s = oracle.render_view(oracle.OracleScene(host, values="bf16"), cam, order, mlp, pixels=pix)
        assert np.abs(got - r_s).max() <= TOL, v
        r_m, _, _ = oracle.render_view(oracle.OracleScene(host), cam, order, mlp, pixels=pix)
        assert psnr(got, r_m) >= 45.0 and np.abs(got - r_m).max() <= 1e-2, v
        assert (n_s > 0).mean() > 0.2, v


# ---------------------------------------------------------------------------
# 2^20 random rays over 2x2 FP32 blocks (the differentiation benchmark)


def test_fit_2x2_full_launch_sampled_rays():
    sc, _, o, d, mlp, _ = synth.workload_grad(device="cuda")
    n = o.shape[0]
    assert n == 1 << 20
    ids = [0, 1, 2, 3]
    ctx = cow.Context(sc, "fp32")
    mlp_d = torch.from_numpy(mlp).cuda()
    rgb, aux, ns = ctx.render_rays(o, d, ids, mlp_d, nsamp=True)
    rng = np.random.default_rng(21)
    pick = np.unique(np.concatenate([rng.integers(0, n, 120), [0, n - 1]]))
    sel = torch.from_numpy(pick).cuda()
    g = np.zeros((n, 3), np.float32)
    g[pick] = rng.normal(size=(len(pick), 3)).astype(np.float32)
    gg = [torch.zeros(b.grid.shape, device="cuda") for b in sc.blocks]
    gp = [[torch.zeros(p.shape, device="cuda") for p in b.planes] for b in sc.blocks]
    gm = torch.zeros(499, device="cuda")
    ctx.render_backward(o, d, ids, mlp_d, aux, torch.from_numpy(g).cuda(), gg, gp, gm)
    ctx.sync_check()
    ctx.close()
    host = synth.Scene([b.to("cpu") for b in sc.blocks], sc.box_lo, sc.box_hi)
    osc = oracle.OracleScene(host)
    o_s, d_s = o[sel].cpu(), d[sel].cpu()
    r_o, a_o, n_o = oracle.render_rays(osc, ids, o_s, d_s, mlp)
    assert np.array_equal(ns[sel].cpu().numpy(), n_o)
    assert (n_o > 0).mean() > 0.5
    assert np.abs(rgb[sel].cpu().numpy() - r_o).max() <= TOL
    assert np.abs(aux[sel].cpu().numpy() - a_o).max() <= TOL
    og, op, om = oracle.render_rays_grad(osc, ids, o_s, d_s, mlp, g[pick])
    for b in range(4):
        if np.abs(og[b]).max() > 0:
            assert_grad(gg[b].cpu().numpy(), og[b], str(("grid", b)))
        else:
            assert float(gg[b].abs().max()) == 0.0, ("grid", b)
        for k in range(3):
            if np.abs(op[b][k]).max() > 0:
                assert_grad(gp[b][k].cpu().numpy(), op[b][k], str(("plane", b, k)))
            else:
                assert float(gp[b][k].abs().max()) == 0.0, ("plane", b, k)
    assert_grad(gm.cpu().numpy(), om, "mlp")
    assert sum(np.count_nonzero(x) for x in og) > 1000
