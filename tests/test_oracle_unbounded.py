"""Pins of the oracle's unbounded boundary blocks (MERF scene contraction,
Eq. 16, Implementation Details): the contraction itself at textbook points,
the closed-form number of recurrence steps to the far limit (one lattice
step of the dominant contracted coordinate per step), an independent numpy
float32 / float64 re-statement of whole rays, and the block-sequential ==
single-pass equivalence (Appendix A) with contracted blocks."""
import math

import numpy as np
import torch

from paper_2312_16457_gb300 import synth

F32 = np.float32


def test_contract_special_values(orc):
    np.testing.assert_array_equal(orc.contract([0.3, -0.5, 1.0]), [0.3, -0.5, 1.0])
    np.testing.assert_allclose(orc.contract([3.0, 1.5, -0.5]), [2 - 1 / 3, 0.5, -1 / 6], rtol=0, atol=1e-15)
    np.testing.assert_allclose(orc.contract([-4.0, 4.0, 1.0]), [-1.75, 1.75, 0.25], rtol=0, atol=1e-15)
    assert abs(orc.contract([1e6, 0.0, 0.0])[0] - 2.0) < 1e-5


def _const_unbounded(P, sigma=0.5, R=9):
    g = torch.zeros(R, R, R, 8)
    g[..., 0] = math.log(sigma)
    planes = [torch.zeros(P, P, 8) for _ in range(3)]
    b = synth.Block((-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), R, P, 1, -1, g, planes,
                    synth.CONTRACTED | synth.EXT_XLO | synth.EXT_XHI | synth.EXT_YLO | synth.EXT_YHI)
    return synth.Scene([b], (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0))


def _shell_steps(delta, x0, xmax=1e4):
    """Steps of x <- x + delta max(1, x)^2 from x0 until x > xmax, in FP64:
    w = 1/x falls by delta w / (w + delta) per step -- by about delta while
    w >> delta (the continuous (1/delta)(1 - 1/xmax)), then geometrically."""
    n, x = 0, x0
    while x <= xmax:
        n += 1
        x += delta * max(1.0, x) ** 2
    return n


def test_step_count_to_the_far_limit(orc):
    """From the centre along an axis: P/2 lattice steps to the box face, then
    the recurrence's count to ||x|| = 1e4 (a handful more than the continuous
    (P/2)(1 - 1e-4)); the steps are delta inside and delta x^2 outside."""
    P = 64
    osc = orc.OracleScene(_const_unbounded(P))
    delta = 2.0 / P
    for d in ([1.0, 0.0, 0.0], [0.0, -1.0, 0.0], [0.0, 0.0, 1.0]):
        o = np.zeros(3, np.float32)
        dd = np.asarray(d, np.float32)
        t, blk, _ = orc.ray_samples(osc, [0], o, dd)
        st = orc.ray_sample_steps(osc, [0], o, dd)
        n_in = int((t < 1.0).sum())
        n_out = len(t) - n_in
        assert abs(n_in - P / 2) <= 1
        want = _shell_steps(delta, float(t[n_in - 1]) + delta) + 1
        assert abs(n_out - want) <= 1, (n_in, n_out, want)
        assert P / 2 <= n_out <= P / 2 + 8  # a linear-in-x step would take ~(P/2) ln(1e4) = 295
        x = np.abs(t)  # |x| = t / h with h = 1 along an axis
        np.testing.assert_allclose(st, delta * np.maximum(1.0, x) ** 2, rtol=1e-6)
        assert np.all(np.diff(t) > 0)


def _np_march(osc, sc, order, o, d):
    """Independent re-statement: FP32 decisions (membership, recurrence,
    contraction, occupancy cell), FP64 interpolation and compositing."""
    o = o.astype(F32)
    d = d.astype(F32)
    samples = []
    for k in order:
        b = sc.blocks[k]
        lo, hi = np.asarray(b.lo, F32), np.asarray(b.hi, F32)
        ext = b.unbounded
        delta = F32((float(b.hi[0]) - float(b.lo[0])) / b.P)

        def owned(p):
            return ((ext & 1) or p[0] >= lo[0]) and ((ext & 2) or p[0] < hi[0]) and \
                   ((ext & 4) or p[1] >= lo[1]) and ((ext & 8) or p[1] < hi[1])

        i, limit = 0, 1 << 15  # far enough for the rays of this camera to reach every region they cross
        while i < limit and not owned(o + (F32(i) + F32(0.5)) * delta * d):
            i += 1
        if i == limit:
            continue
        t = (F32(i) + F32(0.5)) * delta
        c = np.asarray([(float(b.lo[a]) + float(b.hi[a])) / 2 for a in range(3)], F32)
        ih = np.asarray([2.0 / (float(b.hi[a]) - float(b.lo[a])) for a in range(3)], F32)
        bits = osc.occ[k]
        nc = -(-(b.R - 1) // sc.occ_cell)
        kk = F32((b.R - 1) / 4.0)
        for _ in range(65536):
            p = o + t * d
            if not owned(p):
                break
            x = (p - c) * ih
            m = np.abs(x).max()
            if m > F32(1e4):
                break
            m1 = max(m, F32(1.0))
            step = (delta * m1) * m1
            if m <= 1:
                u = x.copy()
            else:
                u = np.where(np.abs(x) == m, np.sign(x) * (F32(2.0) - F32(1.0) / np.abs(x)), x / m).astype(F32)
            v = np.clip(np.floor((u + F32(2.0)) * kk).astype(np.int64), 0, b.R - 2)
            cell = v // sc.occ_cell
            ci = (cell[2] * nc + cell[1]) * nc + cell[0]
            if (bits[ci >> 5] >> (ci & 31)) & 1:
                samples.append((float(t), k, float(step), p.astype(np.float64)))
            t = t + step
    return samples


def _feature(b, u):
    """FP64 trilinear + 3 bilinear lookups at contracted coordinates u."""
    g = b.grid.double().numpy()

    def axis(val, n):
        s = min(max((val + 2.0) * (n - 1) / 4.0, 0.0), n - 1.0)
        c0 = min(int(math.floor(s)), n - 2)
        return c0, s - c0

    (x0, fx), (y0, fy), (z0, fz) = (axis(u[a], b.R) for a in range(3))
    f = np.zeros(8)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = (fx if dx else 1 - fx) * (fy if dy else 1 - fy) * (fz if dz else 1 - fz)
                f += w * g[z0 + dz, y0 + dy, x0 + dx]
    for pl, (ua, va) in enumerate(((0, 1), (0, 2), (1, 2))):
        pp = b.planes[pl].double().numpy()
        (u0, fu), (v0, fv) = axis(u[ua], b.P), axis(u[va], b.P)
        for dv in (0, 1):
            for du in (0, 1):
                f += (fu if du else 1 - fu) * (fv if dv else 1 - fv) * pp[v0 + dv, u0 + du]
    return f


def test_unbounded_rays_brute_force(orc):
    sc, cams, _ = synth.workload_unbounded(R=10, P=24, width=8, height=6)
    osc = orc.OracleScene(sc)
    ids = list(range(len(sc.blocks)))
    o, d = orc.pixel_rays(cams[0])
    rgb, aux, ns = orc.render_rays(osc, ids, o, d)
    far = 0
    for r in range(len(o)):
        order = orc.sort_ids_for_ray(osc, ids, o[r])
        smp = _np_march(osc, sc, list(order), o[r], d[r])
        t, blk, _ = orc.ray_samples(osc, order, o[r], d[r])
        assert len(smp) == ns[r] == len(t)
        np.testing.assert_array_equal(t, [s[0] for s in smp])
        np.testing.assert_array_equal(blk, [s[1] for s in smp])
        far += sum(1 for s in smp if s[2] > 4 * (2.0 / 24))
        T, Cd, F = 1.0, np.zeros(3), np.zeros(4)
        for tt, k, step, p in smp:
            b = sc.blocks[k]
            x = np.array([(p[a] - 0.5 * (b.lo[a] + b.hi[a])) / (0.5 * (b.hi[a] - b.lo[a])) for a in range(3)])
            m = np.abs(x).max()
            u = x if m <= 1 else np.where(np.abs(x) == m, np.sign(x) * (2 - 1 / np.abs(x)), x / m)
            f = _feature(b, u)
            a = -math.expm1(-math.exp(f[0]) * step)
            Cd += T * a / (1 + np.exp(-f[1:4]))
            F += T * a / (1 + np.exp(-f[4:8]))
            T *= 1 - a
        np.testing.assert_allclose(aux[r], np.concatenate([Cd, F, [T]]), rtol=0, atol=1e-12)
    assert far > 20  # samples far out in the contracted shell were exercised


def test_block_sequential_equals_single_pass_unbounded(orc):
    sc, cams, _ = synth.workload_unbounded(R=10, P=24, width=16, height=10)
    osc = orc.OracleScene(sc)
    order = orc.sort_view(osc, list(range(len(sc.blocks))), cams[0])
    a0 = orc.render_view(osc, cams[0], order, None, orc.MODE_BLOCKWISE)[1]
    a1 = orc.render_view(osc, cams[0], order, None, orc.MODE_SINGLE_PASS)[1]
    np.testing.assert_allclose(a0, a1, rtol=0, atol=1e-12)
    assert (a0[:, 7] < 0.5).mean() > 0.5  # the horizon is mostly opaque


def test_contraction_golden_points(orc):
    """Eq. 16 at the hand-worked points of tests/golden/contraction_eq16.txt."""
    import pathlib

    rows = [ln.split() for ln in (pathlib.Path(__file__).parent / "golden" / "contraction_eq16.txt").read_text().splitlines()
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) >= 6
    for row in rows:
        v = [float(t) for t in row]
        np.testing.assert_allclose(orc.contract(np.array(v[:3])), v[3:], rtol=0, atol=1e-15)
