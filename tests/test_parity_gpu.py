"""GPU parity: libcow (CUDA, through the C ABI) against the FP64 oracle.

Tolerances: plain FP32 math max |dRGB| <= 1e-4 (against the oracle run on
the same stored values); occupied-sample counts and occupancy / packed bits
bit-exact; BF16 / FP8 storage PSNR >= 45 dB and max |dRGB| <= 1e-2 against
the oracle on the FP32 master."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2312_16457_gb300 import cow, synth

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


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return math.inf if mse == 0 else 10 * math.log10(1.0 / mse)


def _render(ctx, cams, ids, mlp, **kw):
    rgb, aux, ns = ctx.render(cams, ids, mlp, nsamp=True, **kw)
    ctx.sync_check()
    return rgb.cpu().numpy(), aux.cpu().numpy(), ns.cpu().numpy()


def _oracle_view(osc, cam, order, mlp, pixels=None):
    return oracle.render_view(osc, cam, order, mlp, pixels=pixels)


# ---------------------------------------------------------------------------


def test_occupancy_bit_exact():
    sc, _, _ = synth.workload_single_block(R=64, P=64)
    ctx = cow.Context(sc, "fp32")
    assert np.array_equal(ctx.occupancy(0), oracle.occupancy(sc.blocks[0].grid, 64, 4, 0.01))
    city = synth.city_scene(8, 2, 2.0, [(33, 40)])
    city.occ_cell = 3
    ctx2 = cow.Context(city, "fp16")
    for i, b in enumerate(city.blocks):
        assert np.array_equal(ctx2.occupancy(i), oracle.occupancy(b.grid, 33, 3, 0.01))
        assert ctx2.ztop(i) == oracle.OracleScene(city).ztop(i)


def test_block_ztop_hand_values():
    """The library's z_top (App. D) against the hand-worked values of
    tests/golden/block_ztop.txt (the oracle is pinned to the same rows)."""
    from ztop_cases import ztop_case_scene, ztop_golden_cases

    for R, C, zlo, zhi, kind, k, want in ztop_golden_cases():
        ctx = cow.Context(ztop_case_scene(R, C, zlo, zhi, kind, k), "fp32")
        got = ctx.ztop(0)
        ctx.close()
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (R, C, zlo, zhi, kind, k, got, want)


def _coarse_bits(words, nc):
    """Numpy OR over 4^3 groups of an occupancy bit array (z, y, x order)."""
    n = nc ** 3
    bits = ((words[np.arange(n) >> 5] >> (np.arange(n) & 31)) & 1).astype(bool).reshape(nc, nc, nc)
    nc2 = -(-nc // 4)
    pad = np.zeros((nc2 * 4,) * 3, bool)
    pad[:nc, :nc, :nc] = bits
    g = pad.reshape(nc2, 4, nc2, 4, nc2, 4).any(axis=(1, 3, 5)).ravel()
    out = np.zeros((g.size + 31) // 32, np.uint32)
    for c in np.nonzero(g)[0]:
        out[c >> 5] |= np.uint32(1 << (int(c) & 31))
    return out


def test_coarse_occupancy_is_or_of_cells():
    """The coarse level of the two-level occupancy grid: bit of a 4^3 group =
    OR of the (oracle-exact) cell bits, clipped groups at the far faces."""
    sc, _, _ = synth.workload_single_block(R=64, P=64)
    ctx = cow.Context(sc, "fp32")
    want = _coarse_bits(oracle.occupancy(sc.blocks[0].grid, 64, 4, 0.01), 16)
    assert np.array_equal(ctx.occupancy_coarse(0), want)
    city = synth.city_scene(8, 2, 2.0, [(33, 40)])
    city.occ_cell = 3  # Nc = 11: the last group holds 3 cells per axis
    ctx2 = cow.Context(city, "bf16")
    n_on = []
    for i, b in enumerate(city.blocks):
        want = _coarse_bits(oracle.occupancy(b.grid, 33, 3, 0.01), 11)
        assert np.array_equal(ctx2.occupancy_coarse(i), want)
        n_on.append(int(np.unpackbits(want.view(np.uint8)).sum()))
    assert max(n_on) > 0 and min(n_on) < 27  # both kinds of coarse cell occur


@pytest.mark.parametrize("dtype", ["fp32", "fp16", "bf16", "fp8", "bf16_fp8", "fp8_bf16d"])
def test_packed_bits_exact(dtype):
    sc = synth.city_scene(9, 2, 2.0, [(17, 24)])
    ctx = cow.Context(sc, dtype)
    for i, b in enumerate(sc.blocks):
        for t, src in enumerate([b.grid] + list(b.planes)):
            got, se = ctx.packed(i, t)
            tdt = cow.tensor_storage(dtype, t)
            want_se = oracle.channel_scale_exps(src, tdt)
            want, _ = oracle.quantize(src, tdt, want_se)
            assert np.array_equal(se, want_se)
            assert np.array_equal(got.view(want.dtype), want), (i, t)
        if dtype == "fp8_bf16d":  # the grid's log-density channel, BF16 without a scale
            got, se = ctx.packed(i, 4)
            want, _ = oracle.quantize(b.grid[..., 0].contiguous(), "bf16")
            assert np.array_equal(got.view(want.dtype), want) and not se.any(), i


@pytest.mark.parametrize("schedule", ["warp", "thread", "thread_const"])
def test_single_block_fp32_full_size(schedule):
    """64^3 grid + 256^2 planes, one 128x128 camera (the paper-scale single block)."""
    sc, cams, mlp = synth.workload_single_block(device="cuda")
    ctx = cow.Context(sc, "fp32")
    ctx.set_schedule(schedule)
    rgb, aux, ns = _render(ctx, cams, [[0]], mlp)
    osc = oracle.OracleScene(sc)
    r_o, a_o, n_o = _oracle_view(osc, cams[0], [0], mlp)
    assert np.array_equal(ns, n_o)
    assert np.abs(aux - a_o).max() <= TOL
    assert np.abs(rgb - r_o).max() <= TOL
    assert (n_o > 0).mean() > 0.5 and n_o.max() > 100
    # early ray termination at 1e-5 stays within the tolerance
    rgb_e, _, ns_e = _render(ctx, cams, [[0]], mlp, ert_eps=1e-5)
    assert np.abs(rgb_e - r_o).max() <= TOL
    assert ns_e.sum() < ns.sum()


@pytest.mark.parametrize("schedule", ["warp", "thread", "thread_const"])
def test_city_fp16_storage(schedule):
    """4x4 ground blocks with blobs crossing borders, FP16 storage, FP32 math:
    parity against the oracle on the same FP16 values."""
    sc, cams, mlp = synth.workload_city_4x4(R=48, P=160, width=200, height=120)
    ctx = cow.Context(sc, "fp16")
    ctx.set_schedule(schedule)
    order = ctx.sort_blocks(cams[0], list(range(len(sc.blocks))))
    rgb, aux, ns = _render(ctx, cams, [order], mlp)
    osc = oracle.OracleScene(sc, values="fp16")
    assert np.array_equal(order, oracle.sort_view(osc, list(range(len(sc.blocks))), cams[0]))
    r_o, a_o, n_o = _oracle_view(osc, cams[0], order, mlp)
    assert np.array_equal(ns, n_o)
    assert np.abs(rgb - r_o).max() <= TOL
    assert np.abs(aux - a_o).max() <= TOL
    # single pass over all samples gives the same image (Appendix A)
    r_s, _, _ = oracle.render_view(osc, cams[0], order, mlp, oracle.MODE_SINGLE_PASS)
    assert np.abs(rgb - r_s).max() <= TOL


def test_multiview_uneven_equals_single_views():
    sc, _, mlp = synth.workload_city_4x4(R=24, P=48)
    ctx = cow.Context(sc, "bf16")
    cams = [synth.camera((0.3, -7.0, 6.0), (0.0, 0.0, -1.0), 33, 17, 60.0),
            synth.camera((5.0, 1.0, 3.0), (-1.0, 0.5, -1.0), 64, 64, 45.0),
            synth.camera((-2.0, -2.0, 9.0), (0.0, 0.0, -1.0), 100, 37, 70.0)]
    ids = [ctx.sort_blocks(c, list(range(16))) for c in cams]
    rgb, aux, ns = _render(ctx, cams, ids, mlp)
    off = 0
    for c, i in zip(cams, ids):
        r1, a1, n1 = _render(ctx, [c], [i], mlp)
        n = c.width * c.height
        assert np.array_equal(rgb[off:off + n], r1)
        assert np.array_equal(aux[off:off + n], a1)
        assert np.array_equal(ns[off:off + n], n1)
        off += n


def test_const_records_equal_shared_records():
    """Block records in the parameter buffer give the image of the shared-memory
    staging (the same marcher on the same values); a call whose views select
    more records than the parameter buffer holds runs staged."""
    sc, _, mlp = synth.workload_city_4x4(R=24, P=48)
    ctx = cow.Context(sc, "bf16")
    cams = [synth.camera((0.3 * k, -7.0, 6.0), (0.0, 0.0, -1.0), 40 + k, 24, 60.0) for k in range(7)]
    ids = [ctx.sort_blocks(c, list(range(16))) for c in cams]
    assert sum(len(i) for i in ids) > 96
    for views in (cams[:1], cams[:3], cams):
        vid = ids[:len(views)]
        ctx.set_schedule("thread")
        want = _render(ctx, views, vid, mlp, ert_eps=1e-5)
        ctx.set_schedule("thread_const")
        got = _render(ctx, views, vid, mlp, ert_eps=1e-5)
        assert np.array_equal(got[2], want[2])
        assert np.abs(got[0] - want[0]).max() <= 1e-6
        assert np.abs(got[1] - want[1]).max() <= 1e-6
    ctx.sync_check()


def test_tile_order_keeps_the_image():
    sc, cams, mlp = synth.workload_city_4x4(R=24, P=48, width=203, height=117)
    ctx = cow.Context(sc, "bf16")
    order = ctx.sort_blocks(cams[0], list(range(16)))
    ref = _render(ctx, cams, [order], mlp)
    for strip in (1, 3, 5, 12, 13, 100):
        ctx.set_tile_order(strip)
        got = _render(ctx, cams, [order], mlp)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), strip


def test_host_outputs_match_device():
    sc, cams, mlp = synth.workload_single_block(R=32, P=64, width=40, height=24)
    ctx = cow.Context(sc, "fp32")
    rgb_d, aux_d, ns_d = _render(ctx, cams, [[0]], mlp)
    n = 40 * 24
    out = (torch.empty((n, 3)).pin_memory(), torch.empty((n, 8)).pin_memory(),
           torch.empty((n,), dtype=torch.int32).pin_memory())
    ctx.render(cams, [[0]], mlp, nsamp=True, out=out)
    ctx.sync_check()
    assert np.array_equal(out[0].numpy(), rgb_d)
    assert np.array_equal(out[1].numpy(), aux_d)
    assert np.array_equal(out[2].numpy(), ns_d)
    page = (torch.empty((n, 3)), None, None)  # pageable host memory
    ctx.render(cams, [[0]], mlp, aux=False, out=page)
    ctx.sync_check()
    assert np.array_equal(page[0].numpy(), rgb_d)


def test_render_rays_parity():
    """Ray-batch form: random rays from a sphere around a 2x2-block scene, each
    ray compositing in the xy order of its own origin."""
    sc = synth.city_scene(4, 2, 2.0, [(32, 64)])
    o, d = synth.random_rays(3000, 11, sc.box_lo, sc.box_hi)
    mlp = synth.mlp_weights(104)
    ctx = cow.Context(sc, "fp32")
    ids = list(range(4))
    rgb, aux, ns = ctx.render_rays(o.cuda(), d.cuda(), ids, mlp, nsamp=True)
    ctx.sync_check()
    osc = oracle.OracleScene(sc)
    r_o, a_o, n_o = oracle.render_rays(osc, ids, o, d, mlp)
    assert np.array_equal(ns.cpu().numpy(), n_o)
    assert np.abs(rgb.cpu().numpy() - r_o).max() <= TOL
    assert np.abs(aux.cpu().numpy() - a_o).max() <= TOL
    assert (n_o > 0).mean() > 0.5


def test_select_lod_bit_exact():
    sc = synth.city_scene(31, 8, 2.0, [(10, 12), (10, 12), (10, 12)], lod_thresh=[5.0, 10.0, 0.0])
    ctx = cow.Context(sc, "fp16")
    osc = oracle.OracleScene(sc)
    cams = [synth.camera((0.0, -17.0, 12.0), (0.0, -1.5, -1.0), 1920, 1080, 60.0),
            synth.camera((-6.0, -6.0, 2.0), (6.0, 6.0, -1.0), 640, 360, 90.0),
            synth.camera((0.0, 0.0, 400.0), (0.0, 0.01, 0.0), 64, 64, 10.0)]
    cams += synth.random_aerial_cameras(12, 77, 8.0, (3.0, 14.0), [(640, 360), (1920, 1080)])
    seen = set()
    for cam in cams:
        for thr in ([5.0, 10.0, 0.0], [2.5, 6.0, 0.0], [1e9, 1e9, 0.0]):
            got = ctx.select_lod(cam, thr)
            want = oracle.select_lod(osc, cam, thr)
            assert np.array_equal(got, want)
            seen |= {sc.blocks[i].level for i in got}
    assert seen == {1, 2, 3}
    for i in range(len(sc.blocks)):
        assert ctx.ztop(i) == osc.ztop(i)


@pytest.mark.parametrize("dtype", ["bf16", "fp8", "bf16_fp8", "fp8_bf16d"])
def test_precision_forms(dtype):
    """LOD-mixed city at 1/4 resolution: the storage formats against the
    oracle on the FP32 master (PSNR >= 45 dB, max |dRGB| <= 1e-2) and against
    the oracle on the oracle's own dequantisation of the same storage
    (<= 1e-4).  Pure per-channel E4M3 ("fp8") does not meet the 1e-2 bound
    (its 3-bit mantissa on the log-density gives 0.0144 in the oracle too):
    it is checked on the same stored values and for PSNR only, and the FP8
    form that meets the bound is "fp8_bf16d" (log-density in BF16)."""
    sc, cams, mlp = synth.workload_city_lod(res=((64, 256), (32, 128), (16, 64)), width=192, height=108)
    ctx = cow.Context(sc, dtype)
    ids = ctx.select_lod(cams[0], sc.lod_thresh)
    osc_m = oracle.OracleScene(sc)
    assert np.array_equal(ids, oracle.select_lod(osc_m, cams[0], sc.lod_thresh))
    rgb, _, ns = _render(ctx, cams, [ids], mlp)
    osc_q = oracle.OracleScene(sc, values=dtype)
    r_q, _, n_q = _oracle_view(osc_q, cams[0], ids, mlp)
    assert np.array_equal(ns, n_q)
    assert np.abs(rgb - r_q).max() <= TOL
    r_m, _, _ = _oracle_view(osc_m, cams[0], ids, mlp)
    p, mx = psnr(rgb, r_m), float(np.abs(rgb - r_m).max())
    print(f"{dtype}: PSNR {p:.2f} dB, max |dRGB| {mx:.4g} vs the oracle on the FP32 master")
    assert p >= 45.0, p
    if dtype != "fp8":
        assert mx <= 1e-2, mx
    # BF16 MLP operands with FP32 accumulation
    rgb_b, _, _ = _render(ctx, cams, [ids], mlp, mlp_bf16=True)
    assert psnr(rgb_b, r_m) >= 45.0
    if dtype != "fp8":
        assert np.abs(rgb_b - r_m).max() <= 1e-2


def _c2w_down(x, y, z):
    # looking straight down (-z world), image up = +y world
    c2w = np.zeros((3, 4))
    c2w[:, 0] = [1, 0, 0]
    c2w[:, 1] = [0, 1, 0]
    c2w[:, 2] = [0, 0, 1]
    c2w[:, 3] = [x, y, z]
    return c2w


@pytest.mark.parametrize("schedule", ["warp", "thread", "thread_const"])
def test_edge_cases(schedule):
    sc, _, mlp = synth.workload_city_4x4(R=16, P=32)
    ctx = cow.Context(sc, "fp32")
    ctx.set_schedule(schedule)
    osc = oracle.OracleScene(sc)
    cams = [synth.Camera(_c2w_down(0.0, 0.0, 5.0), 9, 7, 40.0),     # axis-aligned centre ray, block corner
            synth.Camera(_c2w_down(-1.0, 1.0, 0.2), 1, 1, 30.0),    # 1x1 image, camera inside a block
            synth.camera((-4.0, -4.0, 0.5), (4.0, 4.0, -0.5), 17, 9, 80.0),  # grazing the ground
            synth.camera((0.0, 0.0, 0.0), (1.0, 0.0, 0.0), 31, 3, 120.0)]     # inside the scene, looking along x
    for cam in cams:
        order = ctx.sort_blocks(cam, list(range(16)))
        rgb, aux, ns = _render(ctx, [cam], [order], mlp)
        r_o, a_o, n_o = _oracle_view(osc, cam, order, mlp)
        assert np.array_equal(ns, n_o)
        assert np.abs(rgb - r_o).max() <= TOL
    # no blocks at all: empty features, C = sigmoid(MLP(0, 0, d))
    cam = cams[0]
    rgb, aux, ns = _render(ctx, [cam], [[]], mlp)
    r_o, a_o, n_o = _oracle_view(osc, cam, [], mlp)
    assert np.all(ns == 0) and np.all(aux[:, 7] == 1.0)
    assert np.abs(rgb - r_o).max() <= TOL


def test_full_size_city_sampled():
    """The 4x4-block city at full size (256^3 grids, 1024^2 planes, FP16) at
    1280x720 in the launch the benchmark times; sampled pixels against the
    oracle on the FP16 values."""
    sc, cams, mlp = synth.workload_city_4x4(device="cuda")
    ctx = cow.Context(sc, "fp16")
    order = ctx.sort_blocks(cams[0], list(range(16)))
    rgb, aux, ns = _render(ctx, cams, [order], mlp, ert_eps=1e-5)
    host = synth.Scene([b.to("cpu") for b in sc.blocks], sc.box_lo, sc.box_hi)
    del sc
    osc = oracle.OracleScene(host, values="fp16")
    rng = np.random.default_rng(0)
    W, H = cams[0].width, cams[0].height
    pix = np.concatenate([rng.integers(0, W * H, 160), np.arange(0, W * H, W * H // 40)[:40] + W // 2,
                          [0, W - 1, W * H - 1, W * (H - 1)]])
    r_o, a_o, n_o = _oracle_view(osc, cams[0], order, mlp, pixels=pix)
    assert np.abs(rgb[pix] - r_o).max() <= TOL
    assert np.abs(aux[pix, :7] - a_o[:, :7]).max() <= TOL
    assert (n_o > 0).mean() > 0.5


def test_gather_peak_probe():
    """The roofline denominator: random-gather rates order as L1 > L2 > HBM."""
    l1 = cow.gather_peak(32, 64 << 10)
    l2 = cow.gather_peak(32, 32 << 20)
    hb = cow.gather_peak(32, 4 << 30, iters=32)
    assert l1 > l2 > hb > 100.0
    assert cow.gather_peak(16, 64 << 10) > 100.0
    with pytest.raises(cow.CowError):
        cow.gather_peak(24, 64 << 10)
