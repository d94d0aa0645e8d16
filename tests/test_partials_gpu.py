"""GPU parity of the block-parallel form: per-block partials
(cow_render_partials) against the oracle's single-block renders, and K2
(cow_composite_over) against the fused ray form and the oracle."""
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


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_partials_and_composite(storage):
    sc = synth.city_scene(23, 2, 2.0, [(24, 40)])
    o, d = synth.random_rays(3000, 5, sc.box_lo, sc.box_hi)
    mlp = synth.mlp_weights(8)
    ids = [0, 1, 2, 3]
    ctx = cow.Context(sc, storage)
    oc, dc = o.cuda(), d.cuda()
    part = ctx.render_partials(oc, dc, ids)
    ctx.sync_check()
    osc = oracle.OracleScene(sc, values="master" if storage == "fp32" else storage)
    pn = part.cpu().numpy()
    for k in ids:  # every partial is its block rendered alone (Eq. 11)
        _, a_o, _ = oracle.render_rays(osc, [k], o, d)
        assert np.abs(pn[:, k, :] - a_o).max() <= TOL, k
    assert (pn[:, :, 7] < 1.0).sum(axis=1).max() >= 2  # rays through several blocks
    mlp_d = torch.from_numpy(mlp).cuda()
    rgb, aux = ctx.composite_over(oc, dc, ids, part, mlp_d)
    ref, ref_aux, _ = ctx.render_rays(oc, dc, ids, mlp_d)
    ctx.sync_check()
    assert float((rgb - ref).abs().max()) <= 1e-5
    assert float((aux - ref_aux).abs().max()) <= 1e-5
    r_o, a_o, _ = oracle.render_rays(osc, ids, o, d, mlp)
    assert np.abs(rgb.cpu().numpy() - r_o).max() <= TOL
    # the blocks split between two calls (a block-space split) composite to the same image
    p01 = ctx.render_partials(oc, dc, [0, 1])
    p23 = ctx.render_partials(oc, dc, [2, 3])
    rgb2, _ = ctx.composite_over(oc, dc, ids, torch.cat([p01, p23], dim=1), mlp_d)
    ctx.sync_check()
    assert torch.equal(rgb2, rgb)
    # BF16 MLP operands: the precision form's bound against the oracle (the
    # operands' BF16 rounding can differ between the two FP32 paths)
    rgb_b, _ = ctx.composite_over(oc, dc, ids, part, mlp_d, mlp_bf16=True)
    ctx.sync_check()
    r_m, _, _ = oracle.render_rays(oracle.OracleScene(sc), ids, o, d, mlp)
    assert np.abs(rgb_b.cpu().numpy() - r_m).max() <= 1e-2
    ctx.close()


def test_partials_unbounded_and_bricks():
    sc, _, mlp = synth.workload_unbounded(R=40, P=48)
    o, d = synth.random_rays(1500, 9, sc.box_lo, sc.box_hi)
    oc, dc = o.cuda(), d.cuda()
    ids = [0, 1, 2, 3]
    mlp_d = torch.from_numpy(mlp).cuda()
    dense = cow.Context(sc, "fp16")
    sparse = cow.Context(sc, "fp16", bricks=True)
    pd = dense.render_partials(oc, dc, ids)
    ps = sparse.render_partials(oc, dc, ids)
    assert torch.equal(pd, ps)
    rgb, _ = dense.composite_over(oc, dc, ids, pd, mlp_d)
    ref, _, _ = dense.render_rays(oc, dc, ids, mlp_d)
    dense.sync_check()
    assert float((rgb - ref).abs().max()) <= 1e-5
    dense.close()
    sparse.close()


def test_partials_arguments():
    sc = synth.city_scene(23, 2, 2.0, [(8, 8)])
    ctx = cow.Context(sc, "fp32")
    o = torch.zeros(4, 3, device="cuda")
    d = torch.zeros(4, 3, device="cuda")
    d[:, 2] = -1.0
    with pytest.raises(cow.CowError):
        ctx.render_partials(o, d, [0, 7])  # id out of range
    with pytest.raises(cow.CowError):
        ctx.render_partials(o, d, list(range(4)) * 17)  # more than 64 ids
    part = ctx.render_partials(o[:0], d[:0], [0])  # an empty batch
    assert part.shape == (0, 1, 8)
    ctx.close()
