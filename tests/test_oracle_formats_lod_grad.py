"""Oracle pins for storage formats, LOD selection (Appendix D) and gradients."""
import math

import numpy as np
import pytest
import torch

from paper_2312_16457_gb300 import synth
from ztop_cases import ztop_case_scene, ztop_golden_cases


# ---------------------------------------------------------------------------
# storage formats against library conversions


def _edge_values():
    rng = np.random.default_rng(1)
    v = np.concatenate([
        rng.normal(size=2000) * 3,
        rng.uniform(-1e-3, 1e-3, 500),
        rng.uniform(-1e-6, 1e-6, 200),
        [0.0, -0.0, 1.0, -1.0, 65504.0, 65519.0, 6.1e-5, 5.96e-8, 2.98e-8, 1e-10],
    ]).astype(np.float32)
    return v


def test_fp16_matches_numpy(orc):
    v = _edge_values()
    want = v.astype(np.float16).view(np.uint16)
    bits, deq = orc.quantize(v, "fp16")
    assert np.array_equal(bits, want)
    assert np.array_equal(deq, v.astype(np.float16).astype(np.float32))


def test_bf16_matches_torch(orc):
    v = _edge_values()
    want = torch.from_numpy(v).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    bits, deq = orc.quantize(v, "bf16")
    assert np.array_equal(bits, want)


def test_e4m3_matches_torch(orc):
    codes = np.arange(256, dtype=np.uint8)
    dec = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    for c in range(256):
        mine = orc.e4m3_value(int(c))
        if np.isnan(dec[c]):
            assert np.isnan(mine)
        else:
            assert mine == dec[c]
    rng = np.random.default_rng(2)
    v = np.concatenate([rng.normal(size=3000) * 40, rng.uniform(-0.02, 0.02, 500),
                        [0.0, 448.0, -448.0, 1.0 / 512, 3.0 / 1024]]).astype(np.float32)
    v = v[np.abs(v) <= 448]
    want = torch.from_numpy(v).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    bits, _ = orc.quantize(v, "fp8")
    assert np.array_equal(bits, want)
    # saturation to the largest finite value
    assert orc.f32_to_e4m3_bits(1000.0) == 0x7E
    assert orc.f32_to_e4m3_bits(-470.0) == 0xFE


def test_e4m3_scale_exponent(orc):
    for amax in [1e-5, 0.3, 1.0, 3.5, 448.0, 448.0001, 897.0, 2e4]:
        e = orc.e4m3_scale_exp(amax)
        assert amax <= 448.0 * 2.0 ** e
        assert amax > 448.0 * 2.0 ** (e - 1)
    x = np.array([[3.0, -12.0, 0.0, 1e-3, 500.0, -7.0, 2.0, 1.0]] * 4, np.float32)
    se = orc.channel_scale_exps(x, "fp8")
    _, deq = orc.quantize(x, "fp8", se)
    # with per-channel scales every channel keeps FP8's 3-bit relative precision
    assert np.all(np.abs(deq.reshape(x.shape) - x) <= np.abs(x) / 16 + 1e-30)


# ---------------------------------------------------------------------------
# LOD selection (Appendix D)


def _lod_scene():
    # 4x4 level-1 blocks of side 2, 2x2 level-2 blocks of side 4, 1 level-3 block
    return synth.city_scene(31, 4, 2.0, [(6, 8), (6, 8), (6, 8)])


def test_lod_block_counts():
    """Sec. 4.1 rendering stage: K / 4^(l-1) blocks at level l, 2x2 merged."""
    sc = _lod_scene()
    K = len(sc.ids_at_level(1))
    for lev in (1, 2, 3):
        assert len(sc.ids_at_level(lev)) == K // 4 ** (lev - 1)
    for i, b in enumerate(sc.blocks):
        if b.parent >= 0:
            p = sc.blocks[b.parent]
            assert p.level == b.level + 1
            assert p.lo[0] <= b.lo[0] and b.hi[0] <= p.hi[0] and p.lo[1] <= b.lo[1] and b.hi[1] <= p.hi[1]


def _dist(orc, osc, i, cam):
    b = osc.scene.blocks[i]
    c = np.array([(b.lo[0] + b.hi[0]) / 2, (b.lo[1] + b.hi[1]) / 2, osc.ztop(i)])
    return float(np.linalg.norm(c - cam.c2w[:, 3]))


def _check_cover(sc, ids):
    """selected footprints are disjoint"""
    for a in range(len(ids)):
        for b in range(a + 1, len(ids)):
            A, B = sc.blocks[ids[a]], sc.blocks[ids[b]]
            ox = min(A.hi[0], B.hi[0]) - max(A.lo[0], B.lo[0])
            oy = min(A.hi[1], B.hi[1]) - max(A.lo[1], B.lo[1])
            assert ox <= 0 or oy <= 0


def test_lod_far_camera_keeps_coarsest(orc):
    sc = _lod_scene()
    osc = orc.OracleScene(sc)
    cam = synth.camera((0.0, 0.0, 500.0), (0.0, 0.01, 0.0), 64, 64, 10.0)
    ids = orc.select_lod(osc, cam, [3.0, 6.0, 0.0])
    assert list(ids) == sc.ids_at_level(3)


def test_lod_near_camera_descends(orc):
    """A camera low over one corner block: that region comes at level 1, the
    far quadrants stay coarse; results are sorted by xy distance."""
    sc = _lod_scene()
    osc = orc.OracleScene(sc)
    cam = synth.camera((-3.0, -3.0, 2.0), (3.0, 3.0, -1.0), 64, 48, 90.0)
    thr = [3.5, 6.5, 0.0]
    ids = orc.select_lod(osc, cam, thr)
    levels = [sc.blocks[i].level for i in ids]
    assert 1 in levels and 2 in levels and 3 not in levels
    _check_cover(sc, ids)
    # a level-1 block is only reached when its parent had a child within the
    # level-1 threshold; a kept level-2 block whose children are all within
    # the camera's view has all of them beyond it
    for i in ids:
        b = sc.blocks[i]
        kids_of_parent = [j for j, c in enumerate(sc.blocks) if c.parent == b.parent]
        if b.level == 1:
            assert min(_dist(orc, osc, j, cam) for j in kids_of_parent) <= thr[0]
        d = [_dist(orc, osc, j, cam) for j, c in enumerate(sc.blocks) if c.parent == i]
        assert all(abs(x - thr[b.level - 2]) > 1e-6 for x in d) if b.level > 1 else True
    # near-to-far xy sort, ties by index
    o = cam.c2w[:, 3]
    keys = [((sc.blocks[i].lo[0] + sc.blocks[i].hi[0]) / 2 - o[0]) ** 2 +
            ((sc.blocks[i].lo[1] + sc.blocks[i].hi[1]) / 2 - o[1]) ** 2 for i in ids]
    assert keys == sorted(keys)
    # the region under the camera is covered by level-1 blocks
    corner = [i for i in ids if sc.blocks[i].lo[0] == -4.0 and sc.blocks[i].lo[1] == -4.0]
    assert len(corner) == 1 and sc.blocks[corner[0]].level == 1


def test_lod_culls_blocks_behind(orc):
    sc = _lod_scene()
    osc = orc.OracleScene(sc)
    up = synth.camera((0.0, 0.0, 5.0), (0.0, 0.001, 50.0), 32, 32, 60.0)  # looking at the sky
    assert len(orc.select_lod(osc, up, [3.0, 6.0, 0.0])) == 0
    side = synth.camera((-6.0, 0.0, 0.0), (-50.0, 0.0, 0.0), 32, 32, 40.0)  # facing away
    assert len(orc.select_lod(osc, side, [3.0, 6.0, 0.0])) == 0
    # a narrow view of one level-1 block when thresholds force level 1
    narrow = synth.camera((-3.0, -3.0, 6.0), (-3.0, -2.99, -1.0), 16, 16, 5.0)
    ids = orc.select_lod(osc, narrow, [100.0, 100.0, 0.0])
    assert len(ids) >= 1 and all(sc.blocks[i].level == 1 for i in ids)
    assert any(sc.blocks[i].lo[0] == -4.0 and sc.blocks[i].lo[1] == -4.0 for i in ids)
    assert len(ids) <= 4


def test_lod_visibility_matches_pixel_rays(orc):
    """Every block that some pixel ray samples is selected (conservative
    visibility never drops a block that contributes)."""
    sc = _lod_scene()
    osc = orc.OracleScene(sc)
    cam = synth.camera((5.5, -1.0, 1.5), (-1.0, 1.5, -1.0), 40, 30, 50.0)
    lvl1 = sc.ids_at_level(1)
    ids = orc.select_lod(osc, cam, [1e9, 1e9, 0.0])  # force level 1
    assert set(ids) <= set(lvl1)
    order = orc.sort_view(osc, lvl1, cam)
    o, d = orc.pixel_rays(cam)
    touched = set()
    for k in range(0, len(o), 7):
        _, blk, _ = orc.ray_samples(osc, order, o[k], d[k])
        touched |= set(blk.tolist())
    assert touched and touched <= set(ids.tolist())


# ---------------------------------------------------------------------------
# gradient: analytic FP64 adjoint vs central finite differences


def test_gradient_matches_finite_differences(orc):
    sc = synth.city_scene(17, 2, 2.0, [(6, 8)])
    osc = orc.OracleScene(sc, values="f64")
    ids = list(range(len(sc.blocks)))
    o, d = synth.random_rays(48, 3, sc.box_lo, sc.box_hi)
    mlp = synth.mlp_weights(8).astype(np.float64)
    g = np.random.default_rng(4).normal(size=(48, 3))

    def loss():
        rgb, _, _ = orc.render_rays(osc, ids, o, d, mlp)
        return float((rgb * g).sum())

    gg, gp, gm = orc.render_rays_grad(osc, ids, o, d, mlp, g)
    rng = np.random.default_rng(5)
    h = 1e-6
    checked = 0
    # (array, gradient) pools: grids, planes, MLP
    pools = [(osc.grids[b], gg[b]) for b in range(len(ids))]
    pools += [(osc.planes[b][p], gp[b][p]) for b in range(len(ids)) for p in range(3)]
    cands = []
    for k, (arr, gr) in enumerate(pools):
        nz = np.flatnonzero(np.abs(gr.reshape(-1)) > 1e-4)
        for j in rng.choice(nz, size=min(6, len(nz)), replace=False):
            cands.append((arr.reshape(-1), gr.reshape(-1), int(j)))
    for j in rng.choice(499, size=16, replace=False):
        cands.append((mlp, gm, int(j)))
    for arr, gr, j in cands[:80]:
        x0 = arr[j]
        arr[j] = x0 + h
        lp = loss()
        arr[j] = x0 - h
        lm = loss()
        arr[j] = x0
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gr[j]) <= 1e-4 * max(abs(fd), 1e-3), (fd, gr[j])
        checked += 1
    assert checked >= 64


# ---------------------------------------------------------------------------
# z_top (Appendix D: the height of the highest part within the block)


def test_block_ztop_hand_values(orc):
    """orc_block_ztop against z_top worked out by hand: an empty block, one
    dense vertex on and off cell boundaries, slabs ending on and inside a
    cell, cell edges 3 and 4, and R - 1 not a multiple of the cell edge (the
    clamp to the top vertex).  A reading of the top as the highest row's
    bottom vertex (c C), or without the clamp, fails several rows."""
    cases = ztop_golden_cases()
    assert len(cases) >= 12
    for R, C, zlo, zhi, kind, k, want in cases:
        osc = orc.OracleScene(ztop_case_scene(R, C, zlo, zhi, kind, k))
        got = osc.ztop(0)
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (R, C, zlo, zhi, kind, k, got, want)
