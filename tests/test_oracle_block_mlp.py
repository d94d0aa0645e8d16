"""Pins of the oracle's per-block deferred-MLP form (Sec. 4.1 rendering
stage: one MLP Phi^{k,l} per block; Sec. 4.2, Eq. 5 with Eq. 3 per block)
and of its multi-frequency PE(d).

Each test fails for a plausible mistake: PE special values catch a wrong
order of sin / cos or octave; the single-block case pins the per-block MLP
to the global form's MLP (a wrong layout of the n_in-input weights); the
Lambertian case is the paper's Appendix A equivalence (a wrong blend weight
or transmittance); the hand-wired MLP checks which input a PE term reaches;
the brute force composes single-block renders by Eq. 5 (a wrong block's MLP
or a transmittance not carried); the empty block pins the reading that a
block without occupied samples takes no part."""
import math

import numpy as np
import pytest
import torch

from paper_2312_16457_gb300 import synth


def _sig(x):
    return 1.0 / (1.0 + np.exp(-x))


def test_param_count_matches_generator(orc):
    for L in (0, 1, 4):
        assert orc.block_mlp_nparam(L) == synth.block_mlp_nparam(L)
        assert orc.pe_dim(L) == 3 + 6 * L
    assert orc.block_mlp_nparam(0) == synth.MLP_NPARAM


def test_pe_special_values(orc):
    """d = (0, pi/2, pi): sin / cos at octaves 1 and 2 take textbook values."""
    d = np.array([0.0, math.pi / 2, math.pi])
    e = orc.pe(d, 2)
    assert e.shape == (15,)
    np.testing.assert_allclose(e[0:3], d, atol=0)
    np.testing.assert_allclose(e[3:6], [0.0, 1.0, 0.0], atol=1e-15)     # sin(d)
    np.testing.assert_allclose(e[6:9], [1.0, 0.0, -1.0], atol=1e-15)    # cos(d)
    np.testing.assert_allclose(e[9:12], [0.0, 0.0, 0.0], atol=1e-15)    # sin(2d)
    np.testing.assert_allclose(e[12:15], [1.0, -1.0, 1.0], atol=1e-15)  # cos(2d)
    assert orc.pe(d, 0).tolist() == d.tolist()


def test_single_block_reduces_to_global_form(orc):
    """One block, L = 0, its MLP equal to the global one: every pixel with an
    occupied sample gets the global form's colour; the others get 0."""
    sc = synth.single_block_scene(1, 24, 64)
    cam = synth.camera((0.0, -2.5, 0.8), (0.0, 0.0, 0.0), 40, 32, 60.0)
    osc = orc.OracleScene(sc)
    mlp = synth.mlp_weights(101)
    r_g, a_g, n_g = orc.render_view(osc, cam, [0], mlp)
    r_b, a_b, n_b = orc.render_view_block_mlp(osc, cam, [0], mlp[None, :], 0)
    assert np.array_equal(n_g, n_b)
    hit = n_g > 0
    assert 0.2 < hit.mean() < 1.0
    np.testing.assert_allclose(r_b[hit], r_g[hit], rtol=0, atol=1e-13)
    assert np.all(r_b[~hit] == 0.0)
    np.testing.assert_allclose(a_b, a_g, rtol=0, atol=1e-13)


def test_lambertian_equals_single_pass(orc):
    """Appendix A: with every block's Phi = 0 (final bias -1e4 makes the
    sigmoid exactly 0) the Eq. 5 blend of per-block colours equals volume
    rendering over all samples of the scene in one pass."""
    sc = synth.city_scene(5, 2, 2.0, [(12, 32)])
    n = len(sc.blocks)
    L = 3
    w = synth.block_mlp_weights(7, n, L).astype(np.float64)
    w[:, -3:] = -1e4
    osc = orc.OracleScene(sc)
    cam = synth.camera((0.4, -4.5, 3.5), (0.0, 0.0, -0.5), 48, 36, 60.0)
    order = orc.sort_view(osc, list(range(n)), cam)
    r_b, a_b, n_b = orc.render_view_block_mlp(osc, cam, order, w, L)
    r_s, a_s, n_s = orc.render_view(osc, cam, order, None, orc.MODE_SINGLE_PASS)
    assert np.array_equal(n_b, n_s)
    assert (n_b > 0).mean() > 0.25
    np.testing.assert_allclose(r_b, r_s, rtol=0, atol=1e-12)
    np.testing.assert_allclose(a_b, a_s, rtol=0, atol=1e-12)


def test_pe_term_reaches_its_input(orc):
    """A hand-wired MLP passes one input through: W1[i][0] = W2[0][0] =
    W3[0][0] = 1, all else 0.  Then Phi_0 = sigmoid(max(x_i, 0)) and
    Phi_1 = Phi_2 = 1/2, with x = [C_d, F, d, sin d, cos d, sin 2d, cos 2d]."""
    sc = synth.single_block_scene(1, 24, 64)
    cam = synth.camera((0.3, -2.5, 0.8), (0.0, 0.0, 0.0), 24, 20, 60.0)
    osc = orc.OracleScene(sc)
    L = 2
    n_in = 10 + 6 * L
    o, d = orc.pixel_rays(cam)
    d = d.astype(np.float64)
    cases = {7: d[:, 0], 8: d[:, 1], 10 + 1: np.sin(d[:, 1]), 10 + 3 + 2: np.cos(d[:, 2]),
             10 + 6 + 0: np.sin(2 * d[:, 0]), 10 + 9 + 1: np.cos(2 * d[:, 1]), 3: None}
    for i, want in cases.items():
        w = np.zeros(synth.block_mlp_nparam(L))
        w[i * 16 + 0] = 1.0                          # W1[i][0]
        w[n_in * 16 + 16 + 0] = 1.0                  # W2[0][0]
        w[n_in * 16 + 16 + 256 + 16 + 0] = 1.0       # W3[0][0]
        rgb, aux, ns = orc.render_view_block_mlp(osc, cam, [0], w[None, :], L)
        hit = ns > 0
        assert hit.mean() > 0.3
        phi = rgb[hit] - aux[hit, :3]
        x = aux[hit, 3] if want is None else want[hit]  # input 3 is F_0
        np.testing.assert_allclose(phi[:, 0], _sig(np.maximum(x, 0.0)), rtol=0, atol=1e-14)
        np.testing.assert_allclose(phi[:, 1:], 0.5, rtol=0, atol=1e-15)


def test_blend_of_single_block_renders(orc):
    """Eq. 5 by brute force: render each block alone (its C^k, 1 - alpha^k)
    and blend near to far in numpy; equals the multi-block render."""
    sc = synth.city_scene(6, 2, 2.0, [(12, 32)])
    n = len(sc.blocks)
    L = 4
    w = synth.block_mlp_weights(8, n, L, spread=0.5)
    osc = orc.OracleScene(sc)
    cam = synth.camera((-0.6, -4.0, 3.0), (0.2, 0.3, -0.5), 40, 30, 70.0)
    order = orc.sort_view(osc, list(range(n)), cam)
    rgb, aux, ns = orc.render_view_block_mlp(osc, cam, order, w, L)
    C = np.zeros_like(rgb)
    T = np.ones(rgb.shape[0])
    nsum = np.zeros_like(ns)
    multi = np.zeros_like(ns)
    for k in order:
        r_k, a_k, n_k = orc.render_view_block_mlp(osc, cam, [k], w, L)
        C += T[:, None] * r_k
        T *= a_k[:, 7]
        nsum += n_k
        multi += n_k > 0
    assert (multi >= 2).mean() > 0.05  # rays that cross a block border with samples on both sides
    assert np.array_equal(ns, nsum)
    np.testing.assert_allclose(rgb, C, rtol=0, atol=1e-13)
    np.testing.assert_allclose(aux[:, 7], T, rtol=0, atol=1e-15)
    # the blocks' MLPs differ: a global MLP on the blended features gives another image
    r_g, _, _ = orc.render_view(osc, cam, order, w[0])
    assert np.abs(r_g - rgb).max() > 1e-2


def test_block_without_samples_takes_no_part(orc):
    """A block the rays cross only through empty cells adds nothing, although
    its MLP on empty features is not zero."""
    sc = synth.city_scene(9, 2, 2.0, [(12, 32)])
    sc.blocks[1].grid[..., 0] = -12.0  # sigma = 6e-6 < the 0.01 occupancy threshold everywhere
    n = len(sc.blocks)
    L = 1
    w = synth.block_mlp_weights(3, n, L)
    osc = orc.OracleScene(sc)
    cam = synth.camera((0.0, -4.0, 3.0), (0.0, 0.0, -0.5), 32, 24, 70.0)
    order = orc.sort_view(osc, list(range(n)), cam)
    assert 1 in list(order)
    rgb, aux, ns = orc.render_view_block_mlp(osc, cam, order, w, L)
    keep = [k for k in order if k != 1]
    rgb2, aux2, ns2 = orc.render_view_block_mlp(osc, cam, keep, w, L)
    assert np.array_equal(ns, ns2)
    assert np.array_equal(rgb, rgb2) and np.array_equal(aux, aux2)
    r1, _, n1 = orc.render_view_block_mlp(osc, cam, [1], w, L)
    assert np.all(n1 == 0) and np.all(r1 == 0.0)


def test_identical_block_mlps_seam_only_where_blocks_meet(orc):
    """The per-block form with the same MLP in every block (L = 0, the global
    MLP's layout) against the global form: a ray whose occupied samples all
    lie in one block gets the same colour (Eq. 5 with one term is Eq. 3),
    while a ray with samples in two or more blocks does not, because the MLP
    is not linear in (C_d, F).  This is the seam of the per-block form for
    view-dependent colour, which the global form does not have."""
    sc = synth.city_scene(6, 2, 2.0, [(12, 32)])
    n = len(sc.blocks)
    mlp = synth.mlp_weights(106)
    w = np.repeat(mlp[None, :].astype(np.float64), n, axis=0)
    osc = orc.OracleScene(sc)
    cam = synth.camera((-0.6, -4.0, 3.0), (0.2, 0.3, -0.5), 40, 30, 70.0)
    order = orc.sort_view(osc, list(range(n)), cam)
    r_b, a_b, n_b = orc.render_view_block_mlp(osc, cam, order, w, 0)
    r_g, a_g, n_g = orc.render_view(osc, cam, order, mlp)
    assert np.array_equal(n_b, n_g)
    np.testing.assert_allclose(a_b, a_g, rtol=0, atol=1e-13)  # the blended C_d, F, T are the same
    blocks_hit = np.zeros_like(n_b)
    for k in order:
        _, _, n_k = orc.render_view_block_mlp(osc, cam, [k], w, 0)
        blocks_hit += n_k > 0
    one = blocks_hit == 1
    many = blocks_hit >= 2
    assert one.mean() > 0.15 and many.mean() > 0.05
    np.testing.assert_allclose(r_b[one], r_g[one], rtol=0, atol=1e-13)
    seam = np.abs(r_b[many] - r_g[many]).max(axis=1)
    assert seam.max() > 1e-2 and np.median(seam) > 1e-4


def test_ray_form_equals_view_form(orc):
    """Independent rays through the pixel centres of a view, each sorting the
    blocks from its own origin (the camera centre), composite exactly as the
    view form does; a ray batch mixing two origins equals its two halves
    rendered apart."""
    sc = synth.city_scene(6, 2, 2.0, [(12, 32)])
    n = len(sc.blocks)
    L = 2
    w = synth.block_mlp_weights(8, n, L, spread=0.5)
    osc = orc.OracleScene(sc)
    cam = synth.camera((-0.6, -4.0, 3.0), (0.2, 0.3, -0.5), 32, 24, 70.0)
    order = orc.sort_view(osc, list(range(n)), cam)
    pix = np.arange(0, 32 * 24, 3)
    r_v, a_v, n_v = orc.render_view_block_mlp(osc, cam, order, w, L, pixels=pix)
    o, d = orc.pixel_rays(cam, pix)
    r_r, a_r, n_r = orc.render_rays_block_mlp(osc, list(range(n)), o, d, w, L)
    assert np.array_equal(n_r, n_v) and (n_v > 0).mean() > 0.3
    np.testing.assert_allclose(r_r, r_v, rtol=0, atol=1e-13)
    np.testing.assert_allclose(a_r, a_v, rtol=0, atol=1e-13)
    o2, d2 = synth.random_rays(64, 5, sc.box_lo, sc.box_hi)
    oo = np.concatenate([o, o2.numpy()])
    dd = np.concatenate([d, d2.numpy()])
    r_m, _, n_m = orc.render_rays_block_mlp(osc, list(range(n)), oo, dd, w, L)
    r_2, _, n_2 = orc.render_rays_block_mlp(osc, list(range(n)), o2, d2, w, L)
    assert np.array_equal(n_m, np.concatenate([n_r, n_2]))
    np.testing.assert_allclose(r_m, np.concatenate([r_r, r_2]), rtol=0, atol=0)


def test_ray_form_gradient_matches_finite_differences(orc):
    """The analytic FP64 adjoint of the per-block form (features and every
    block's MLP) against central differences of the FP64 render."""
    sc = synth.city_scene(17, 2, 2.0, [(6, 8)])
    n = len(sc.blocks)
    L = 2
    osc = orc.OracleScene(sc, values="f64")
    ids = list(range(n))
    o, d = synth.random_rays(48, 3, sc.box_lo, sc.box_hi)
    w = synth.block_mlp_weights(9, n, L, spread=0.3).astype(np.float64)
    g = np.random.default_rng(4).normal(size=(48, 3))

    def loss():
        rgb, _, _ = orc.render_rays_block_mlp(osc, ids, o, d, w, L)
        return float((rgb * g).sum())

    gg, gp, gm = orc.render_rays_block_mlp_grad(osc, ids, o, d, w, L, g)
    rng = np.random.default_rng(5)
    h = 1e-6
    pools = [(osc.grids[b], gg[b]) for b in range(n)]
    pools += [(osc.planes[b][p], gp[b][p]) for b in range(n) for p in range(3)]
    pools += [(w[b], gm[b]) for b in range(n)]
    cands = []
    for arr, gr in pools:
        nz = np.flatnonzero(np.abs(gr.reshape(-1)) > 1e-4)
        for j in rng.choice(nz, size=min(6, len(nz)), replace=False):
            cands.append((arr.reshape(-1), gr.reshape(-1), int(j)))
    checked = 0
    for arr, gr, j in cands:
        x0 = arr[j]
        arr[j] = x0 + h
        lp = loss()
        arr[j] = x0 - h
        lm = loss()
        arr[j] = x0
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gr[j]) <= 1e-4 * max(abs(fd), 1e-3), (fd, gr[j])
        checked += 1
    assert checked >= 80
    # every block's MLP receives a gradient (each block has samples on some ray)
    assert all(np.abs(gm[b]).max() > 0 for b in range(n))


def test_ray_form_gradient_reduces_to_global_form(orc):
    """One block with the global MLP (L = 0): the per-block form's gradient
    equals the global form's on rays that have occupied samples."""
    sc = synth.single_block_scene(1, 10, 16)
    osc = orc.OracleScene(sc)
    mlp = synth.mlp_weights(101).astype(np.float64)
    o, d = synth.random_rays(64, 7, sc.box_lo, sc.box_hi)
    _, _, ns = orc.render_rays(osc, [0], o, d, mlp)
    hit = ns > 0
    assert hit.mean() > 0.5
    o, d = o[hit], d[hit]
    g = np.random.default_rng(2).normal(size=(len(o), 3))
    gg, gp, gm = orc.render_rays_grad(osc, [0], o, d, mlp, g)
    bg, bp, bm = orc.render_rays_block_mlp_grad(osc, [0], o, d, mlp[None, :], 0, g)
    np.testing.assert_allclose(bg[0], gg[0], rtol=0, atol=1e-12)
    for k in range(3):
        np.testing.assert_allclose(bp[0][k], gp[0][k], rtol=0, atol=1e-12)
    np.testing.assert_allclose(bm[0], gm, rtol=0, atol=1e-12)


def test_ray_form_gradient_of_a_block_without_samples_is_zero(orc):
    """R20 in the adjoint: a block the rays cross only through empty cells
    takes no part, so neither its features nor its MLP receive a gradient,
    and dropping it from ids leaves every other gradient unchanged."""
    sc = synth.city_scene(9, 2, 2.0, [(8, 16)])
    sc.blocks[1].grid[..., 0] = -12.0  # below the occupancy threshold everywhere
    n = len(sc.blocks)
    L = 1
    w = synth.block_mlp_weights(3, n, L)
    osc = orc.OracleScene(sc)
    o, d = synth.random_rays(128, 11, sc.box_lo, sc.box_hi)
    g = np.random.default_rng(6).normal(size=(128, 3))
    gg, gp, gm = orc.render_rays_block_mlp_grad(osc, list(range(n)), o, d, w, L, g)
    assert np.all(gg[1] == 0.0) and all(np.all(x == 0.0) for x in gp[1]) and np.all(gm[1] == 0.0)
    keep = [k for k in range(n) if k != 1]
    gg2, gp2, gm2 = orc.render_rays_block_mlp_grad(osc, keep, o, d, w, L, g)
    for b in keep:  # the oracle sums over rays on several threads: equal up to rounding order
        np.testing.assert_allclose(gg2[b], gg[b], rtol=0, atol=1e-13)
        np.testing.assert_allclose(gm2[b], gm[b], rtol=0, atol=1e-12)
    assert max(np.abs(gg[b]).max() for b in keep) > 0
