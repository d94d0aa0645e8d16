"""Pins of the oracle's training-stage regularisers (Sec. 4.3): the sparsity
loss of Eq. 7 and the block-opacity loss of Eq. 8, with their gradients.

Closed forms on a constant-density block catch a wrong alpha, delta, mean or
entropy; central finite differences in FP64 catch a wrong gradient (a dropped
factor, a wrong tap or sign); the gradients must not touch channels 1-7."""
import math

import numpy as np
import pytest
import torch

from paper_2312_16457_gb300 import synth


def _const_block(lo, hi, R, P, sigma):
    g = torch.zeros(R, R, R, 8)
    g[..., 0] = math.log(sigma)
    g[..., 1:] = 0.3
    planes = [torch.zeros(P, P, 8) for _ in range(3)]
    return synth.Block(tuple(lo), tuple(hi), R, P, 1, -1, g, planes)


def _H(a):
    a = np.clip(a, 1e-6, 1 - 1e-6)
    return -(a * np.log(a) + (1 - a) * np.log(1 - a))


def test_sparsity_closed_form(orc):
    lo, hi = (-1.0, -1.0, -0.5), (1.0, 1.0, 0.5)
    blk = _const_block(lo, hi, 5, 16, 4.0)
    sc = synth.Scene([blk], lo, hi)
    osc = orc.OracleScene(sc)
    pts = np.random.default_rng(1).uniform(-1.5, 1.5, size=(5000, 3)).astype(np.float32)
    loss, gg, gp = orc.sparsity_loss_grad(osc, [0], pts, weight=0.05)
    lo32, hi32 = np.float32(lo), np.float32(hi)
    inside = ((pts[:, :2] >= lo32[:2]) & (pts[:, :2] < hi32[:2])).all(1) & (pts[:, 2] >= lo32[2]) & (pts[:, 2] <= hi32[2])
    sigma = math.exp(float(blk.grid[0, 0, 0, 0]))
    delta = float(np.float32(2.0) / np.float32(16))
    alpha = -math.expm1(-sigma * delta)
    assert 0.1 < inside.mean() < 0.5
    assert loss == pytest.approx(0.05 * inside.mean() * alpha, rel=1e-12)
    # gradient: sum over all taps of d loss / d f0 = weight * mean(inside) * sigma delta (1 - alpha) * (grid + 3 planes)
    total = gg[0][..., 0].sum() + sum(p[..., 0].sum() for p in gp[0])
    assert total == pytest.approx(0.05 * inside.mean() * sigma * delta * (1 - alpha) * 4, rel=1e-10)
    assert np.all(gg[0][..., 1:] == 0) and all(np.all(p[..., 1:] == 0) for p in gp[0])


def test_opacity_closed_form(orc):
    lo, hi = (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)
    blk = _const_block(lo, hi, 5, 32, 0.8)
    sc = synth.Scene([blk], lo, hi)
    osc = orc.OracleScene(sc)
    o, d = synth.random_rays(400, 2, lo, hi)
    loss, _, _ = orc.opacity_loss_grad(osc, [0], o, d, weight=0.001, grad=False)
    _, _, ns = orc.render_rays(osc, [0], o, d)
    sigma = math.exp(float(blk.grid[0, 0, 0, 0]))
    delta = float(np.float32(2.0) / np.float32(32))
    a = 1 - np.exp(-sigma * delta * ns[ns > 0])
    assert (ns > 0).mean() > 0.5 and 0.2 < a.mean() < 0.9
    assert loss == pytest.approx(0.001 * _H(a).sum() / len(ns), rel=1e-10)


@pytest.mark.parametrize("which", ["sparsity", "opacity"])
def test_gradient_matches_finite_differences(orc, which):
    sc = synth.city_scene(23, 2, 2.0, [(6, 8)])
    osc = orc.OracleScene(sc, values="f64")
    ids = list(range(len(sc.blocks)))
    if which == "sparsity":
        pts = np.random.default_rng(7).uniform(np.float32(sc.box_lo), np.float32(sc.box_hi), size=(3000, 3))

        def run(grad=True):
            return orc.sparsity_loss_grad(osc, ids, pts.astype(np.float32), weight=0.7, grad=grad)
    else:
        o, d = synth.random_rays(64, 5, sc.box_lo, sc.box_hi)

        def run(grad=True):
            return orc.opacity_loss_grad(osc, ids, o, d, weight=0.3, grad=grad)

    loss0, gg, gp = run()
    assert loss0 > 0
    pools = [(osc.grids[b], gg[b]) for b in range(len(ids))]
    pools += [(osc.planes[b][p], gp[b][p]) for b in range(len(ids)) for p in range(3)]
    rng = np.random.default_rng(9)
    h = 1e-6
    checked = 0
    for arr, gr in pools:
        flat, gflat = arr.reshape(-1), gr.reshape(-1)
        assert np.all(gr[..., 1:] == 0)  # only the density channel
        nz = np.flatnonzero(np.abs(gflat) > 1e-7)
        for j in rng.choice(nz, size=min(5, len(nz)), replace=False):
            x0 = flat[j]
            flat[j] = x0 + h
            lp = run(False)[0]
            flat[j] = x0 - h
            lm = run(False)[0]
            flat[j] = x0
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gflat[j]) <= 1e-4 * max(abs(fd), 1e-5), (fd, gflat[j])
            checked += 1
    assert checked >= 40
