"""Batched form (one persistent launch over a (view, tile, block) queue):
every pixel has the per-view kernel's occupied samples (bit for bit) and its
colour up to FP32 rounding (the two kernels inline the same code but the
compiler may fuse multiply-adds differently), for every tile shape, with and
without CUDA-graph replay and after autotuning; one view is also checked
against the FP64 oracle directly."""
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


def _scene():
    sc = synth.city_scene(31, 8, 2.0, [(16, 40), (12, 24), (8, 16)], lod_thresh=[5.0, 10.0, 0.0])
    cams = synth.random_aerial_cameras(9, 12, 8.0, (3.0, 14.0), [(96, 54), (64, 64), (40, 23), (131, 77)])
    cams.append(synth.camera((0.0, -9.0, 6.0), (0.0, 0.0, -1.0), 57, 33, 60.0))
    return sc, cams, synth.mlp_weights(7)


@pytest.mark.parametrize("storage", ["bf16", "fp32"])
def test_batch_equals_per_view(storage):
    sc, cams, mlp = _scene()
    ctx = cow.Context(sc, storage)
    ids = [ctx.select_lod(c, sc.lod_thresh) for c in cams]
    mlp_d = torch.from_numpy(mlp).cuda()
    ref = ctx.render(cams, ids, mlp_d, nsamp=True)  # no early termination: sample sets must match exactly
    ref_ert = ctx.render(cams, ids, mlp_d, ert_eps=1e-5, aux=False)[0]
    ctx.sync_check()
    b = cow.Batch(ctx, 16, 4096)
    n = b.set_views(cams, ids)
    assert n == sum(c.width * c.height for c in cams)
    for cfg in range(5):  # 4: warp items
        for graph in (False, True):
            b.set_config(cfg, 3)
            out = (torch.full((n, 3), -1.0, device="cuda"), torch.zeros((n, 8), device="cuda"),
                   torch.zeros(n, dtype=torch.int32, device="cuda"))
            for _ in range(2):
                b.render(mlp_d, *out, graph=graph)
            ctx.sync_check()
            assert torch.equal(out[2], ref[2]), (cfg, graph)
            for k in range(2):
                diff = float((out[k] - ref[k]).abs().max())
                assert diff <= 2e-6, (cfg, graph, k, diff)
    t, c, ms = b.tune(mlp_d, torch.empty((n, 3), device="cuda"), ert_eps=1e-5)
    assert t in range(5) and c in (2, 3, 4, 6, 8) and ms > 0
    out = torch.empty((n, 3), device="cuda")
    b.render(mlp_d, out, ert_eps=1e-5, graph=True)
    ctx.sync_check()
    assert float((out - ref_ert).abs().max()) <= 1e-4  # early termination changes each channel by <= eps
    b.close()


def test_batch_view_against_oracle():
    sc, cams, mlp = _scene()
    ctx = cow.Context(sc, "fp32")
    cam = cams[-1]
    ids = ctx.select_lod(cam, sc.lod_thresh)
    b = cow.Batch(ctx, 1, 256)
    n = b.set_views([cam], [ids])
    out = (torch.empty((n, 3), device="cuda"), None, torch.empty(n, dtype=torch.int32, device="cuda"))
    b.render(torch.from_numpy(mlp).cuda(), out[0], None, out[2])
    ctx.sync_check()
    osc = oracle.OracleScene(sc)
    r_o, _, n_o = oracle.render_view(osc, cam, ids, mlp)
    assert np.array_equal(out[2].cpu().numpy(), n_o)
    assert np.abs(out[0].cpu().numpy() - r_o).max() <= 1e-4


def test_batch_rejects_bad_arguments():
    sc, cams, mlp = _scene()
    ctx = cow.Context(sc, "fp32")
    b = cow.Batch(ctx, 2, 8)
    with pytest.raises(cow.CowError):
        b.set_views(cams[:3], [[0]] * 3)  # more views than the batch holds
    with pytest.raises(cow.CowError):
        b.set_views(cams[:1], [list(range(9))])  # more ids than the batch holds
    with pytest.raises(cow.CowError):
        b.set_config(7, 2)
    # warp items read records from the parameter buffer only
    ctx2 = cow.Context(sc, "bf16")
    b2 = cow.Batch(ctx2, 2, 256)
    n2 = b2.set_views(cams[:2], [ctx2.select_lod(c, sc.lod_thresh) for c in cams[:2]])
    b2.set_config(4, 4)
    b2.set_records("shared")
    with pytest.raises(cow.CowError, match="parameter buffer"):
        b2.render(torch.from_numpy(mlp).cuda(), torch.empty((n2, 3), device="cuda"))
    b2.close()
    ctx2.close()


def test_batch_runs_and_long_lists():
    """Views whose blocks together exceed one launch's parameter buffer (96
    records) are served in several runs, and a view with more than 96
    blocks falls back to records read from memory; both equal the per-view
    kernel (sample counts bit for bit)."""
    sc = synth.city_scene(33, 12, 1.0, [(10, 16)])
    nb = len(sc.blocks)
    ctx = cow.Context(sc, "bf16")
    mlp_d = torch.from_numpy(synth.mlp_weights(5)).cuda()
    cams = [synth.camera((x, y, 2.5), (x + 0.5, y + 0.8, -0.8), 48, 36, 70.0)
            for x, y in ((-4.5, -4.5), (3.0, -4.0), (-4.0, 3.5), (3.5, 3.0))]
    ids = []
    for c in cams:  # each view: the 60 blocks nearest to its camera, near to far
        order = ctx.sort_blocks(c, list(range(nb)))
        ids.append(ctx.sort_blocks(c, sorted(order[:60].tolist())))
    assert len(set(np.concatenate(ids).tolist())) > 96
    cams.append(synth.camera((0.0, -7.0, 4.0), (0.0, 0.0, -0.5), 64, 40, 70.0))
    ids.append(ctx.sort_blocks(cams[-1], list(range(nb))))  # 144 blocks: over 96
    ref = ctx.render(cams, ids, mlp_d, nsamp=True)
    ctx.sync_check()
    b = cow.Batch(ctx, 8, 1024)
    n = b.set_views(cams, ids)
    for graph in (False, True):
        out = (torch.full((n, 3), -1.0, device="cuda"), torch.zeros((n, 8), device="cuda"),
               torch.zeros(n, dtype=torch.int32, device="cuda"))
        b.render(mlp_d, *out, graph=graph)
        ctx.sync_check()
        assert torch.equal(out[2], ref[2]), graph
        assert float((out[0] - ref[0]).abs().max()) <= 2e-6
    # without the long view: every list fits, the views go in runs
    b2 = cow.Batch(ctx, 8, 1024)
    n2 = b2.set_views(cams[:4], ids[:4])
    ref2 = ctx.render(cams[:4], ids[:4], mlp_d, nsamp=True)
    out = (torch.empty((n2, 3), device="cuda"), torch.zeros((n2, 8), device="cuda"),
           torch.zeros(n2, dtype=torch.int32, device="cuda"))
    b2.render(mlp_d, *out, graph=True)
    ctx.sync_check()
    assert torch.equal(out[2], ref2[2])
    assert float((out[0] - ref2[0]).abs().max()) <= 2e-6
    b.close()
    b2.close()


def test_tuners_pick_valid_schedules():
    """cow_tune_schedule (per-view schedule and tile order) and the record
    placement cow_batch_tune adds: the kept configuration is one of the
    candidates and renders the same image."""
    sc, cams, mlp = _scene()
    ctx = cow.Context(sc, "bf16")
    ids = [ctx.select_lod(c, sc.lod_thresh) for c in cams]
    mlp_d = torch.from_numpy(mlp).cuda()
    ref = ctx.render(cams, ids, mlp_d, nsamp=True)
    n = ref[0].shape[0]
    sched, strip, ms = ctx.tune_schedule(cams, ids, mlp_d, torch.empty((n, 3), device="cuda"))
    assert sched in ("thread_const", "thread", "warp") and strip in (0, 2, 4) and ms > 0
    got = ctx.render(cams, ids, mlp_d, nsamp=True)
    ctx.sync_check()
    assert torch.equal(got[2], ref[2])
    assert float((got[0] - ref[0]).abs().max()) <= 2e-6
    b = cow.Batch(ctx, 16, 4096)
    b.set_views(cams, ids)
    for mode in ("shared", "param"):
        b.set_records(mode)
        out = torch.empty((n, 3), device="cuda")
        ns = torch.zeros(n, dtype=torch.int32, device="cuda")
        b.render(mlp_d, out, None, ns, graph=True)
        ctx.sync_check()
        assert torch.equal(ns, ref[2]), mode
    b.tune(mlp_d, torch.empty((n, 3), device="cuda"))
    tile, ctas, rec = b.config()
    assert tile in cow.Batch.TILE_SHAPES.values() and ctas in (2, 3, 4, 6, 8) and rec in ("param", "shared")
    b.close()
    ctx.close()


def test_grid_schedule_equals_per_view():
    """The grid schedule (the view marcher on groups of views whose lists
    fit one parameter buffer; a view over 96 blocks alone) writes the
    per-view render's pixels at each view's place in the batch (sample counts
    bit for bit, colours to FP32 rounding), and the tuner keeps one of the
    two schedules."""
    sc = synth.city_scene(33, 12, 1.0, [(10, 16)])
    nb = len(sc.blocks)
    ctx = cow.Context(sc, "bf16")
    mlp_d = torch.from_numpy(synth.mlp_weights(5)).cuda()
    cams = [synth.camera((x, y, 2.5), (x + 0.5, y + 0.8, -0.8), 48, 36, 70.0)
            for x, y in ((-4.5, -4.5), (3.0, -4.0), (-4.0, 3.5), (3.5, 3.0))]
    ids = []
    for c in cams:
        order = ctx.sort_blocks(c, list(range(nb)))
        ids.append(ctx.sort_blocks(c, sorted(order[:30].tolist())))
    cams.append(synth.camera((0.0, -7.0, 4.0), (0.0, 0.0, -0.5), 64, 40, 70.0))
    ids.append(ctx.sort_blocks(cams[-1], list(range(nb))))  # 144 blocks: a group of its own
    ref = ctx.render(cams, ids, mlp_d, nsamp=True)
    ctx.sync_check()
    b = cow.Batch(ctx, 8, 1024)
    n = b.set_views(cams, ids)
    b.set_schedule("grid")
    assert b.schedule() == "grid"
    out = (torch.full((n, 3), -1.0, device="cuda"), torch.zeros((n, 8), device="cuda"),
           torch.zeros(n, dtype=torch.int32, device="cuda"))
    for graph in (False, True):
        b.render(mlp_d, *out, graph=graph)
        ctx.sync_check()
        assert torch.equal(out[2], ref[2]), graph
        for k in range(2):  # the reference's 264 records go through the shared-memory kernel
            assert float((out[k] - ref[k]).abs().max()) <= 2e-6, (graph, k)
    assert b.last_groups() == 3  # views 0-2 (90 ids), view 3 (30 + 144 > 96), the long view
    b.tune(mlp_d, torch.empty((n, 3), device="cuda"))
    assert b.schedule() in ("queue", "grid")
    out2 = torch.empty((n, 3), device="cuda")
    ns2 = torch.zeros(n, dtype=torch.int32, device="cuda")
    b.render(mlp_d, out2, None, ns2, graph=True)
    ctx.sync_check()
    assert torch.equal(ns2, ref[2])
    assert float((out2 - ref[0]).abs().max()) <= 2e-6
    b.close()
    ctx.close()


@pytest.mark.parametrize("sched", ["queue", "grid"])
def test_batch_view_without_blocks(sched):
    """A view whose block list is empty (nothing selected) renders the empty
    ray's colour, in both schedules, as the per-view render does."""
    sc, cams, mlp = _scene()
    ctx = cow.Context(sc, "bf16")
    ids = [ctx.select_lod(cams[0], sc.lod_thresh), np.zeros(0, np.int32), ctx.select_lod(cams[2], sc.lod_thresh)]
    views = [cams[0], cams[1], cams[2]]
    mlp_d = torch.from_numpy(mlp).cuda()
    ref = ctx.render(views, ids, mlp_d, nsamp=True)
    ctx.sync_check()
    b = cow.Batch(ctx, 4, 512)
    n = b.set_views(views, ids)
    b.set_schedule(sched)
    out = (torch.full((n, 3), -1.0, device="cuda"), torch.zeros((n, 8), device="cuda"),
           torch.zeros(n, dtype=torch.int32, device="cuda"))
    b.render(mlp_d, *out)
    ctx.sync_check()
    assert torch.equal(out[2], ref[2])
    for k in range(2):
        assert float((out[k] - ref[k]).abs().max()) <= 2e-6, k
    p0 = cams[0].width * cams[0].height
    p1 = p0 + cams[1].width * cams[1].height
    assert int(out[2][p0:p1].sum()) == 0
    b.close()
    ctx.close()
