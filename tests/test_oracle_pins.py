"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test would fail for a plausible mistake in the oracle: a wrong alpha
formula or step (closed form), a transposed axis or plane (affine field), a
wrong blend (Appendix A equivalence, negative control), a wrong sample set or
cell rule (independent numpy brute force), a wrong ray (re-projection)."""
import math

import numpy as np
import pytest
import torch

from paper_2312_16457_gb300 import synth


def _const_block(lo, hi, R, P, sigma, c, s):
    g = torch.zeros(R, R, R, 8)
    g[..., 0] = math.log(sigma)
    for k in range(3):
        g[..., 1 + k] = math.log(c[k] / (1 - c[k]))
    for k in range(4):
        g[..., 4 + k] = math.log(s[k] / (1 - s[k]))
    planes = [torch.zeros(P, P, 8) for _ in range(3)]
    return synth.Block(tuple(lo), tuple(hi), R, P, 1, -1, g, planes)


def _slab(o, d, lo, hi):
    t0, t1 = 0.0, math.inf
    for a in range(3):
        if d[a] == 0:
            if not (lo[a] <= o[a] <= hi[a]):
                return None
            continue
        u, v = (lo[a] - o[a]) / d[a], (hi[a] - o[a]) / d[a]
        t0, t1 = max(t0, min(u, v)), min(t1, max(u, v))
    return (t0, t1) if t0 < t1 else None


def test_closed_form_constant_block(orc):
    """Eq. 1-2 and Eq. 13: in a block of constant sigma and colour, n samples
    give T = exp(-sigma delta n), C_d = c (1 - T), F = s (1 - T), and
    n delta approximates the chord length within a step at each end."""
    sigma, c, s = 3.0, (0.2, 0.5, 0.7), (0.1, 0.3, 0.6, 0.9)
    lo, hi = (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)
    blk = _const_block(lo, hi, 6, 32, sigma, c, s)
    sc = synth.Scene([blk], lo, hi)
    osc = orc.OracleScene(sc)
    cam = synth.camera((0.3, -3.0, 1.2), (0.0, 0.0, 0.0), 40, 30, 50.0)
    rgb, aux, ns = orc.render_view(osc, cam, [0])
    delta = float(np.float32(2.0 / 32))
    # the block stores float32 pre-activations: use the values they encode
    g = blk.grid[0, 0, 0].double().numpy()
    sigma = math.exp(g[0])
    c = 1 / (1 + np.exp(-g[1:4]))
    s = 1 / (1 + np.exp(-g[4:8]))
    T = aux[:, 7]
    assert np.allclose(T, np.exp(-sigma * delta * ns), rtol=1e-12, atol=0)
    assert np.allclose(aux[:, :3], np.outer(1 - T, c), rtol=1e-12, atol=1e-15)
    assert np.allclose(aux[:, 3:7], np.outer(1 - T, s), rtol=1e-12, atol=1e-15)
    assert np.array_equal(rgb, aux[:, :3])  # no MLP: C = C_d
    o, d = orc.pixel_rays(cam)
    exact = 0
    for k in range(len(ns)):
        iv = _slab(o[k].astype(np.float64), d[k].astype(np.float64), lo, hi)
        L = 0.0 if iv is None else iv[1] - iv[0]
        assert abs(ns[k] * delta - L) <= 2 * delta + 1e-9
        if iv is not None:
            n_exp = math.floor(iv[1] / delta - 0.5) - math.ceil(iv[0] / delta - 0.5) + 1
            exact += int(n_exp == ns[k])
        else:
            exact += int(ns[k] == 0)
    assert exact >= 0.99 * len(ns)
    assert (ns > 0).sum() > 0.5 * len(ns)


def test_affine_field_exact(orc):
    """Trilinear / bilinear interpolation reproduces affine fields exactly, on
    a non-cubic block so that any axis or plane mix-up shows."""
    rng = np.random.default_rng(7)
    lo, hi = (-1.0, -0.5, -2.0), (1.5, 2.0, 0.5)
    R, P = 5, 7
    A = rng.normal(size=(8, 3))
    e = rng.normal(size=8)
    B, D, E = rng.normal(size=(8, 2)), rng.normal(size=(8, 2)), rng.normal(size=(8, 2))

    def ax(n, a):
        return lo[a] + np.arange(n) * (hi[a] - lo[a]) / (n - 1)

    z, y, x = np.meshgrid(ax(R, 2), ax(R, 1), ax(R, 0), indexing="ij")
    grid = np.stack([A[c, 0] * x + A[c, 1] * y + A[c, 2] * z + e[c] for c in range(8)], -1)
    v, u = np.meshgrid(ax(P, 1), ax(P, 0), indexing="ij")
    pxy = np.stack([B[c, 0] * u + B[c, 1] * v for c in range(8)], -1)
    v, u = np.meshgrid(ax(P, 2), ax(P, 0), indexing="ij")
    pxz = np.stack([D[c, 0] * u + D[c, 1] * v for c in range(8)], -1)
    v, u = np.meshgrid(ax(P, 2), ax(P, 1), indexing="ij")
    pyz = np.stack([E[c, 0] * u + E[c, 1] * v for c in range(8)], -1)
    blk = synth.Block(lo, hi, R, P, 1, -1, torch.from_numpy(grid), [torch.from_numpy(p) for p in (pxy, pxz, pyz)])
    osc = orc.OracleScene(synth.Scene([blk], lo, hi), values="f64")
    pts = rng.uniform(lo, hi, size=(200, 3))
    pts[:5] = [[ax(R, 0)[1], ax(R, 1)[2], ax(R, 2)[3]], lo, hi, [lo[0], hi[1], lo[2]], [hi[0], lo[1], hi[2]]]
    for p in pts:
        want = A @ p + e + B @ p[[0, 1]] + D @ p[[0, 2]] + E @ p[[1, 2]]
        got = orc.feature_at(osc, 0, p)
        assert np.allclose(got, want, rtol=0, atol=1e-12), (p, got - want)


def _tiny_city(M, R=8, P=16, seed=11):
    return synth.city_scene(seed, M, 2.0, [(R, P)])


@pytest.mark.parametrize("M", [2, 4])
def test_block_sequential_equals_single_pass(orc, M):
    """Appendix A: compositing per block (Eq. 11) and across blocks in depth
    order (Eq. 12) equals single-pass volume rendering over all samples
    (Eq. 14), for C_d, F and T; with one global deferred MLP the colours agree
    as well."""
    sc = _tiny_city(M)
    osc = orc.OracleScene(sc)
    cam = synth.camera((0.5, -2.5 * M, 1.5 * M), (0.0, 0.0, -1.0), 32, 32, 60.0)
    order = orc.sort_view(osc, list(range(len(sc.blocks))), cam)
    mlp = synth.mlp_weights(5)
    r0, a0, n0 = orc.render_view(osc, cam, order, mlp, orc.MODE_BLOCKWISE)
    r1, a1, n1 = orc.render_view(osc, cam, order, mlp, orc.MODE_SINGLE_PASS)
    assert np.array_equal(n0, n1)
    assert np.abs(a0 - a1).max() <= 1e-12
    assert np.abs(r0 - r1).max() <= 1e-12
    assert (a0[:, 7] < 0.5).mean() > 0.2  # the rays do hit content


def test_alpha_normalised_blend_fails(orc):
    """Table 4 "no alpha blending": blending blocks by alpha^k / sum alpha^j is
    not volume rendering; it must differ from the single pass."""
    sc = _tiny_city(4)
    osc = orc.OracleScene(sc)
    cam = synth.camera((0.5, -10.0, 6.0), (0.0, 0.0, -1.0), 24, 24, 60.0)
    order = orc.sort_view(osc, list(range(len(sc.blocks))), cam)
    _, a1, _ = orc.render_view(osc, cam, order, None, orc.MODE_SINGLE_PASS)
    _, a2, _ = orc.render_view(osc, cam, order, None, orc.MODE_ALPHA_NORM)
    assert np.abs(a1[:, :7] - a2[:, :7]).max() > 1e-2


def test_depth_sort_is_traversal_order(orc):
    """Appendix D sorts blocks by xy distance of their centres to the camera;
    on a uniform ground grid this is the order in which each ray meets them, so
    the block-sequential sample sequence is in increasing depth."""
    sc = _tiny_city(4)
    osc = orc.OracleScene(sc)
    cam = synth.camera((1.3, -9.0, 5.0), (0.2, 0.0, -1.0), 24, 16, 70.0)
    order = orc.sort_view(osc, list(range(len(sc.blocks))), cam)
    o, d = orc.pixel_rays(cam)
    seen_multi = 0
    for k in range(len(o)):
        t, blk, _ = orc.ray_samples(osc, order, o[k], d[k])
        assert np.all(np.diff(t) > 0)
        seen_multi += int(len(set(blk.tolist())) > 1)
    assert seen_multi > 20


def _np_brute_ray(sc, occ, o, d, mlp):
    """Independent single pass: scan every lattice index, assign the sample to
    the block whose half-open footprint holds it (Eq. 4), look its cell up,
    interpolate with numpy and composite in depth order."""
    f32 = np.float32
    b0 = sc.blocks[0]
    delta = f32((b0.hi[0] - b0.lo[0]) / b0.P)
    # far bound of the whole scene
    iv = _slab(o.astype(np.float64), d.astype(np.float64), np.array(sc.box_lo) - 0.01, np.array(sc.box_hi) + 0.01)
    T, Cd, F = 1.0, np.zeros(3), np.zeros(4)
    n = 0
    if iv is not None:
        for i in range(0, int(iv[1] / float(delta)) + 3):
            t = (f32(i) + f32(0.5)) * delta
            p = o + t * d  # float32 elementwise, no fused multiply-add
            hit = None
            for bi, b in enumerate(sc.blocks):
                lo, hi = np.array(b.lo, f32), np.array(b.hi, f32)
                if lo[0] <= p[0] < hi[0] and lo[1] <= p[1] < hi[1] and lo[2] <= p[2] <= hi[2]:
                    hit = bi
            if hit is None:
                continue
            b = sc.blocks[hit]
            lo, hi = np.array(b.lo, f32), np.array(b.hi, f32)
            k = np.array([f32((b.R - 1) / (float(hi[a]) - float(lo[a]))) for a in range(3)], f32)
            v = np.clip(np.floor((p - lo) * k).astype(int), 0, b.R - 2)
            nc = -(-(b.R - 1) // sc.occ_cell)
            cell = v // sc.occ_cell
            ci = (cell[2] * nc + cell[1]) * nc + cell[0]
            if not (occ[hit][ci >> 5] >> (ci & 31)) & 1:
                continue
            n += 1
            pd = p.astype(np.float64)
            g = np.clip((pd - lo) * (b.R - 1) / (hi.astype(np.float64) - lo), 0, b.R - 1)
            c0 = np.minimum(np.floor(g).astype(int), b.R - 2)
            fr = g - c0
            G = b.grid.numpy().astype(np.float64)
            f = np.zeros(8)
            for dz in (0, 1):
                for dy in (0, 1):
                    for dx in (0, 1):
                        w = (fr[0] if dx else 1 - fr[0]) * (fr[1] if dy else 1 - fr[1]) * (fr[2] if dz else 1 - fr[2])
                        f += w * G[c0[2] + dz, c0[1] + dy, c0[0] + dx]
            h = np.clip((pd - lo) * (b.P - 1) / (hi.astype(np.float64) - lo), 0, b.P - 1)
            h0 = np.minimum(np.floor(h).astype(int), b.P - 2)
            hf = h - h0
            for pl, (ua, va) in enumerate(((0, 1), (0, 2), (1, 2))):
                Pp = b.planes[pl].numpy().astype(np.float64)
                for dv in (0, 1):
                    for du in (0, 1):
                        w = (hf[ua] if du else 1 - hf[ua]) * (hf[va] if dv else 1 - hf[va])
                        f += w * Pp[h0[va] + dv, h0[ua] + du]
            sig = math.exp(f[0])
            alpha = -math.expm1(-sig * float(delta))
            wgt = T * alpha
            Cd += wgt / (1 + np.exp(-f[1:4]))
            F += wgt / (1 + np.exp(-f[4:8]))
            T *= 1 - alpha
    x = torch.tensor(np.concatenate([Cd, F, d.astype(np.float64)]))
    W = torch.tensor(np.asarray(mlp, np.float64))
    h1 = torch.relu(x @ W[0:160].view(10, 16) + W[160:176])
    h2 = torch.relu(h1 @ W[176:432].view(16, 16) + W[432:448])
    out = torch.sigmoid(h2 @ W[448:496].view(16, 3) + W[496:499])
    return Cd + out.numpy(), np.concatenate([Cd, F, [T]]), n


def test_numpy_brute_force(orc):
    sc = _tiny_city(2, R=6, P=12, seed=21)
    osc = orc.OracleScene(sc)
    cam = synth.camera((0.7, -4.5, 3.0), (0.0, 0.0, -1.0), 12, 10, 60.0)
    order = orc.sort_view(osc, list(range(len(sc.blocks))), cam)
    mlp = synth.mlp_weights(9)
    rgb, aux, ns = orc.render_view(osc, cam, order, mlp)
    o, d = orc.pixel_rays(cam)
    hits = 0
    for k in range(0, len(o), 3):
        r, a, n = _np_brute_ray(sc, osc.occ, o[k], d[k], mlp)
        assert n == ns[k]
        assert np.abs(a - aux[k]).max() <= 1e-12
        assert np.abs(r - rgb[k]).max() <= 1e-12
        hits += int(n > 0)
    assert hits > 10


def test_invariants(orc):
    """T in [0, 1], weights sum to 1 - T, 0 <= C_d, F <= 1 - T per channel."""
    sc, cams, mlp = synth.workload_single_block(R=16, P=32, width=48, height=48)
    osc = orc.OracleScene(sc)
    _, aux, ns = orc.render_view(osc, cams[0], [0])
    T = aux[:, 7]
    assert np.all((T >= 0) & (T <= 1))
    assert np.all(aux[:, :7] >= 0)
    assert np.all(aux[:, :7] <= (1 - T)[:, None] + 1e-12)
    o, d = orc.pixel_rays(cams[0], [48 * 24 + 24])
    _, _, al = orc.ray_samples(osc, [0], o[0], d[0])
    assert np.all((al >= 0) & (al < 1))
    w = np.cumprod(np.concatenate([[1.0], 1 - al]))[:-1] * al
    assert abs(w.sum() - (1 - np.prod(1 - al))) < 1e-12


def test_mlp_matches_torch_float64(orc):
    """Eq. 3's deferred MLP equals float64 torch matmuls on the documented
    input-major weight layout."""
    W = synth.mlp_weights(3).astype(np.float64)
    x = np.random.default_rng(0).normal(size=(64, 10))
    got = orc.mlp(W, x)
    Wt = torch.tensor(W)
    xt = torch.tensor(x)
    h1 = torch.relu(xt @ Wt[0:160].view(10, 16) + Wt[160:176])
    h2 = torch.relu(h1 @ Wt[176:432].view(16, 16) + Wt[432:448])
    want = torch.sigmoid(h2 @ Wt[448:496].view(16, 3) + Wt[496:499]).numpy()
    assert np.abs(got - want).max() < 1e-14


def test_pixel_ray_reprojects_to_pixel_centre(orc):
    cam = synth.camera((0.3, -2.0, 1.1), (0.1, 0.2, -0.3), 37, 23, 55.0)
    pix = np.arange(cam.width * cam.height)
    o, d = orc.pixel_rays(cam)
    Rm, t = cam.c2w[:, :3], cam.c2w[:, 3]
    f = 0.5 * cam.height / math.tan(0.5 * math.radians(cam.fov_y_deg))
    assert np.allclose(o, t.astype(np.float32))
    assert np.allclose(np.linalg.norm(d.astype(np.float64), axis=1), 1.0, atol=1e-6)
    pc = (d.astype(np.float64)) @ Rm  # camera-frame directions
    assert np.all(pc[:, 2] < 0)
    x = f * pc[:, 0] / -pc[:, 2] + 0.5 * cam.width
    y = -f * pc[:, 1] / -pc[:, 2] + 0.5 * cam.height
    assert np.abs(x - (pix % cam.width + 0.5)).max() < 1e-3
    assert np.abs(y - (pix // cam.width + 0.5)).max() < 1e-3


def test_occupancy_brute_force(orc):
    rng = np.random.default_rng(3)
    for R, Cc in ((9, 4), (10, 4), (17, 4), (12, 3)):
        g = rng.normal(size=(R, R, R, 8)).astype(np.float32) * 4 - 7
        bits = orc.occupancy(g, R, Cc, 0.01)
        nc = orc.occ_cells(R, Cc)
        hot = g[..., 0] > math.log(0.01)
        for cz in range(nc):
            for cy in range(nc):
                for cx in range(nc):
                    sl = tuple(slice(c * Cc, min(c * Cc + Cc, R - 1) + 1) for c in (cz, cy, cx))
                    want = bool(hot[sl].any())
                    ci = (cz * nc + cy) * nc + cx
                    assert bool((bits[ci >> 5] >> (ci & 31)) & 1) == want


def test_occupancy_single_vertex(orc):
    """A single dense vertex marks exactly the cells whose vertex range holds
    it: two cells per axis on an interior cell boundary, one elsewhere."""
    R, Cc = 13, 4
    nc = orc.occ_cells(R, Cc)
    for v in [(0, 0, 0), (4, 5, 6), (8, 8, 12), (3, 4, 7)]:
        g = np.full((R, R, R, 8), -20.0, np.float32)
        g[v[2], v[1], v[0], 0] = 0.0
        bits = orc.occupancy(g, R, Cc, 0.01)
        per_axis = [[c for c in range(nc) if c * Cc <= x <= c * Cc + Cc] for x in v]
        want = {(cz * nc + cy) * nc + cx for cx in per_axis[0] for cy in per_axis[1] for cz in per_axis[2]}
        got = {i for i in range(nc ** 3) if (bits[i >> 5] >> (i & 31)) & 1}
        assert got == want
