"""Brick-sparse grids (cow_load_blocks_ex with COW_LOAD_BRICKS) against the
dense grids of the same storage format, through the C ABI.

Lattice samples lie in occupied cells, whose bricks are stored, and the
lookup reads the same stored values in the same order, so every output
equals the dense context's bit for bit (gradients, which are scattered with
float atomics, within FP32 summation-order noise); the dense path itself is
checked against the oracle in the other parity tests.  Scenes use the sparse
city generator setting (content in the lower part of the height), with a
grid of R = 40 vertices: 3 bricks per axis, the last one partial."""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_16457_gb300 import cow, synth

pytestmark = pytest.mark.gpu

FORMATS = ["fp32", "fp16", "bf16", "fp8", "bf16_fp8", "fp8_bf16d"]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2312_16457_gb300 import build

    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _scene(R=40, P=48, M=2, seed=11, **kw):
    return synth.city_scene(seed, M, 2.0, [(R, P)], **{**synth.SPARSE_CITY, **kw})


def _cams(sc):
    return [synth.camera((-2.5, -3.0, 2.2), (0.3, 0.4, -0.8), 61, 37, 60.0),
            synth.camera((1.9, 0.3, 0.1), (-2.0, -0.4, -0.6), 23, 45, 75.0),
            synth.Camera(np.array([[1.0, 0, 0, 0.1], [0, 1.0, 0, -0.3], [0, 0, 1.0, 3.0]]), 17, 17, 40.0)]


def _render(ctx, cams, ids, mlp, **kw):
    rgb, aux, ns = ctx.render(cams, ids, mlp, nsamp=True, **kw)
    ctx.sync_check()
    return rgb, aux, ns


def _stored_bricks(ctx, i, R):
    """Bricks with an occupied cell, counted from the exported coarse level."""
    nc = -(-(R - 1) // 4)
    nc2 = -(-nc // 4)
    words = ctx.occupancy_coarse(i)
    n = nc2 ** 3
    return int(((words[np.arange(n) >> 5] >> (np.arange(n) & 31)) & 1).sum())


@pytest.mark.parametrize("storage", FORMATS)
def test_bricks_equal_dense_views(storage):
    sc = _scene()
    mlp = synth.mlp_weights(31)
    dense = cow.Context(sc, storage)
    sparse = cow.Context(sc, storage, bricks=True)
    cams = _cams(sc)
    ids = [dense.sort_blocks(c, list(range(len(sc.blocks)))) for c in cams]
    for schedule in ("warp", "thread", "thread_const"):
        dense.set_schedule(schedule)
        sparse.set_schedule(schedule)
        for ert in (0.0, 1e-5):
            a = _render(dense, cams, ids, mlp, ert_eps=ert)
            b = _render(sparse, cams, ids, mlp, ert_eps=ert)
            for x, y in zip(a, b):
                assert torch.equal(x, y), (storage, schedule, ert)
    assert int(a[2].sum()) > 1000
    # some bricks are empty air (at R = 40 the 16-voxel bricks overhang the
    # 39-voxel grid, so a block may still take more bytes than its dense grid;
    # the full-size sparse city stores far fewer)
    stored = [_stored_bricks(sparse, i, 40) for i in range(len(sc.blocks))]
    assert min(stored) > 0 and min(stored) < 27, stored
    dense.close()
    sparse.close()


@pytest.mark.parametrize("storage", ["bf16", "fp8_bf16d"])
def test_bricks_against_oracle(storage):
    """The brick-sparse render against the oracle on the same stored values
    (<= 1e-4), sample counts bit-exact."""
    sc = _scene()
    mlp = synth.mlp_weights(31)
    ctx = cow.Context(sc, storage, bricks=True)
    osc = oracle.OracleScene(sc, values=storage)
    for cam in _cams(sc)[:2]:
        order = ctx.sort_blocks(cam, list(range(len(sc.blocks))))
        rgb, aux, ns = _render(ctx, [cam], [order], mlp)
        r_o, a_o, n_o = oracle.render_view(osc, cam, order, mlp)
        assert np.array_equal(ns.cpu().numpy(), n_o)
        assert np.abs(rgb.cpu().numpy() - r_o).max() <= 1e-4
        assert np.abs(aux.cpu().numpy()[:, :7] - a_o[:, :7]).max() <= 1e-4
    ctx.close()


@pytest.mark.parametrize("storage", FORMATS)
def test_brick_bytes(storage):
    """Device bytes of a brick-sparse block: its stored bricks (the layout's
    elements per brick: 17^3 FP32 vertices, 16 x 17 x 17 vertex pairs, 16 x 16
    x 17 FP8 quads plus 16^3 density octets) plus the dense planes."""
    sc = _scene()
    ctx = cow.Context(sc, storage, bricks=True)
    dense = cow.Context(sc, storage)
    elem = {"fp32": 32, "fp16": 32, "bf16": 32, "fp8": 16, "bf16_fp8": 32, "fp8_bf16d": 32}[storage]
    dims = {"fp32": 17 * 17 * 17, "fp8_bf16d": 16 * 16 * 17}.get(storage, 16 * 17 * 17)
    R = 40
    for i, b in enumerate(sc.blocks):
        plane_bytes = dense.block_bytes(i) - R ** 3 * elem * (1.5 if storage == "fp8_bf16d" else 1)
        n = _stored_bricks(ctx, i, R)
        grid = n * dims * elem + (n * 4096 * 16 if storage == "fp8_bf16d" else 0)
        assert ctx.block_bytes(i) == grid + plane_bytes, (i, n)
    ctx.close()
    dense.close()


def test_bricks_ray_form_and_gradient():
    sc = _scene(R=40, P=40)
    o, d = synth.random_rays(8192, 12, sc.box_lo, sc.box_hi)
    o, d = o.cuda(), d.cuda()
    mlp = torch.from_numpy(synth.mlp_weights(8)).cuda()
    ids = list(range(4))
    g = torch.from_numpy(np.random.default_rng(3).normal(size=(8192, 3)).astype(np.float32)).cuda()
    out = []
    for bricks in (False, True):
        ctx = cow.Context(sc, "fp32", bricks=bricks)
        rgb, aux, ns = ctx.render_rays(o, d, ids, mlp, nsamp=True)
        gg = [torch.zeros(b.grid.shape, device="cuda") for b in sc.blocks]
        gp = [[torch.zeros(p.shape, device="cuda") for p in b.planes] for b in sc.blocks]
        gm = torch.zeros(499, device="cuda")
        ctx.render_backward(o, d, ids, mlp, aux, g, gg, gp, gm)
        ctx.sync_check()
        out.append((rgb, aux, ns, gg, gp, gm))
        ctx.close()
    (r0, a0, n0, gg0, gp0, gm0), (r1, a1, n1, gg1, gp1, gm1) = out
    assert torch.equal(r0, r1) and torch.equal(a0, a1) and torch.equal(n0, n1)
    assert int(n0.sum()) > 10000

    def close(x, y):
        s = float(y.abs().max())
        return float((x - y).abs().max()) <= 1e-5 * max(s, 1e-30)

    assert close(gm1, gm0)
    for b in range(4):
        assert close(gg1[b], gg0[b]), b
        for k in range(3):
            assert close(gp1[b][k], gp0[b][k]), (b, k)


def test_bricks_batch_and_residency():
    """The persistent batched form and loads under a residency budget on a
    brick-sparse context equal the dense context's per-view renders."""
    sc = _scene(M=4, R=34, P=40, seed=13)
    mlp = torch.from_numpy(synth.mlp_weights(9)).cuda()
    cams = [synth.camera((-4.0, -4.5, 3.0), (0.5, 0.5, -0.8), 48, 32, 60.0),
            synth.camera((3.5, -2.0, 2.0), (-0.5, 1.0, -0.9), 40, 40, 60.0),
            synth.camera((0.0, 4.0, 2.5), (0.0, -1.0, -0.9), 64, 24, 60.0)]
    dense = cow.Context(sc, "bf16")
    sparse = cow.Context(sc, "bf16", bricks=True)
    nb = len(sc.blocks)
    ids = [dense.sort_blocks(c, list(range(nb))) for c in cams]
    ref = _render(dense, cams, ids, mlp)
    batch = cow.Batch(sparse, len(cams), sum(len(i) for i in ids))
    npix = batch.set_views(cams, ids)
    rgb = torch.empty((npix, 3), device="cuda")
    aux = torch.empty((npix, 8), device="cuda")
    ns = torch.empty((npix,), dtype=torch.int32, device="cuda")
    batch.render(mlp, rgb, aux, ns)
    sparse.sync_check()
    assert torch.equal(rgb, ref[0]) and torch.equal(aux, ref[1]) and torch.equal(ns, ref[2])
    batch.close()
    # under a budget that holds about a third of the blocks: loads on demand
    need = max(sum(sparse.block_bytes(i) for i in v) for v in ids)
    sparse.set_residency(max(need, sum(sparse.block_bytes(i) for i in range(nb)) // 3))
    for k, cam in enumerate(cams):
        r = _render(sparse, [cam], [ids[k]], mlp)
        offs = np.concatenate([[0], np.cumsum([c.width * c.height for c in cams])])
        for x, y in zip(r, ref):
            assert torch.equal(x, y[offs[k]:offs[k + 1]]), k
    sparse.set_residency(0)
    dense.close()
    sparse.close()


def test_bricks_update_features_and_block_mlps():
    """Re-packing new features keeps the brick set (occupancy is held fixed)
    and matches the dense context re-packed the same way; the per-block MLP
    form (Eq. 5) reads bricks as well."""
    sc = _scene()
    mlp = synth.mlp_weights(31)
    dense = cow.Context(sc, "bf16")
    sparse = cow.Context(sc, "bf16", bricks=True)
    g = sc.blocks[1].grid.clone()
    g[..., 1:] += 0.25
    pl = [p.clone() * 2.0 for p in sc.blocks[1].planes]
    dense.update_features(1, g, pl)
    sparse.update_features(1, g, pl)
    cams = _cams(sc)[:2]
    ids = [dense.sort_blocks(c, list(range(4))) for c in cams]
    for x, y in zip(_render(dense, cams, ids, mlp), _render(sparse, cams, ids, mlp)):
        assert torch.equal(x, y)
    bm = synth.block_mlp_weights(7, 4, 2)
    dense.set_block_mlps(bm, 2)
    sparse.set_block_mlps(bm, 2)
    for x, y in zip(_render(dense, cams, ids, None, block_mlps=True), _render(sparse, cams, ids, None, block_mlps=True)):
        assert torch.equal(x, y)
    dense.close()
    sparse.close()


def test_bricks_unbounded_blocks():
    sc, cams, mlp = synth.workload_unbounded(R=40, P=48, width=48, height=27)
    dense = cow.Context(sc, "fp16")
    sparse = cow.Context(sc, "fp16", bricks=True)
    ids = [dense.sort_blocks(cams[0], list(range(4)))]
    a = _render(dense, cams, ids, mlp)
    b = _render(sparse, cams, ids, mlp)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    assert int(a[2].sum()) > 0
    dense.close()
    sparse.close()


def test_bricks_refusals():
    sc = _scene()
    ctx = cow.Context(sc, "bf16", bricks=True)
    pts = torch.zeros(16, 3, device="cuda")
    with pytest.raises(cow.CowError, match="brick"):
        ctx.sparsity_loss(pts, [0, 1, 2, 3])
    with pytest.raises(cow.CowError, match="brick"):
        ctx.packed(0, 0)
    ctx.packed(0, 1)  # the planes stay dense
    ctx.close()
    with pytest.raises(cow.CowError, match="occ_cell"):
        cow.Context(sc, "bf16", occ_cell=3, bricks=True)
