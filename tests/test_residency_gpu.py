"""Dynamic loading / unloading under a device-memory budget (App. D) and the
residency-aware view order: images rendered with blocks loaded on demand
equal the all-resident images bit for bit, the bytes loaded equal the
planner's prediction, and the budget is never exceeded."""
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
    sc, _, mlp = synth.workload_batch(res=((16, 64), (8, 32), (4, 16)), n_views=1)
    cams = synth.random_aerial_cameras(12, 21, 16.0, (6.0, 14.0), [(96, 54), (64, 64)])
    return sc, cams, mlp


def test_loaded_on_demand_equals_all_resident():
    sc, cams, mlp = _scene()
    ref = cow.Context(sc, "bf16")
    ctx = cow.Context(sc, "bf16")
    ids = [ref.select_lod(c, sc.lod_thresh) for c in cams]
    want = [ref.render([c], [i], mlp, nsamp=True) for c, i in zip(cams, ids)]
    bb = [ctx.block_bytes(i) for i in range(len(sc.blocks))]
    need = [sum(bb[i] for i in set(v.tolist())) for v in ids]
    budget = int(1.25 * max(need))
    assert budget < sum(bb)  # not everything fits: blocks must be unloaded
    order, planned, given = cow.plan_view_order(bb, [v.tolist() for v in ids], budget)
    ctx.set_residency(budget)
    r0 = ctx.residency()
    assert r0["resident_bytes"] == 0 and r0["resident_blocks"] == 0
    for v in order:
        rgb, aux, ns = ctx.render([cams[v]], [ids[v]], mlp, nsamp=True)
        ctx.sync_check()
        assert ctx.residency()["resident_bytes"] <= budget
        for g, w in zip((rgb, aux, ns), want[v]):
            assert torch.equal(g, w)
    r = ctx.residency()
    assert r["upload_bytes"] - r0["upload_bytes"] == planned
    assert r["evictions"] > r0["evictions"] and planned < sum(need)
    # back to all resident
    ctx.set_residency(0)
    assert ctx.residency()["resident_blocks"] == len(sc.blocks)
    for v in range(3):
        assert torch.equal(ctx.render([cams[v]], [ids[v]], mlp)[0], want[v][0])


def test_over_budget_call_fails_cleanly():
    sc, cams, mlp = _scene()
    ctx = cow.Context(sc, "fp16")
    ids = ctx.select_lod(cams[0], sc.lod_thresh)
    need = sum(ctx.block_bytes(i) for i in set(ids.tolist()))
    ctx.set_residency(need - 1)
    with pytest.raises(cow.CowError) as e:
        ctx.render([cams[0]], [ids], mlp)
    assert e.value.status == 3  # OOM
    assert ctx.residency()["resident_bytes"] <= need - 1
    half = ids[: len(ids) // 2]
    rgb = ctx.render([cams[0]], [half], mlp)[0]
    ctx.sync_check()
    ctx.set_residency(0)
    assert torch.equal(rgb, ctx.render([cams[0]], [half], mlp)[0])


def test_updated_features_survive_unloading():
    """cow_update_features on a loaded block marks it changed: unloading copies
    the new features back, so reloading renders them."""
    sc, cams, mlp = _scene()
    ctx = cow.Context(sc, "fp32")
    ref = cow.Context(sc, "fp32")
    ids = [ref.select_lod(c, sc.lod_thresh) for c in cams]
    k = int(ids[0][0])
    b = sc.blocks[k]
    g2, p2 = b.grid.clone(), [p * 0.5 + 0.05 for p in b.planes]
    ref.update_features(k, g2, p2)
    bb = [ctx.block_bytes(i) for i in range(len(sc.blocks))]
    budget = int(1.25 * max(sum(bb[i] for i in set(v.tolist())) for v in ids))
    ctx.set_residency(budget)
    ctx.render([cams[0]], [ids[0]], mlp)
    ctx.update_features(k, g2, p2)
    ctx.set_residency(1)  # unload every block, block k with its new features
    assert ctx.residency()["resident_blocks"] == 0
    ctx.set_residency(budget)
    for v in range(1, len(cams)):
        ctx.render([cams[v]], [ids[v]], mlp)
    ctx.sync_check()
    got = ctx.render([cams[0]], [ids[0]], mlp)[0]
    assert torch.equal(got, ref.render([cams[0]], [ids[0]], mlp)[0])
    # the packed export of an unloaded block comes from the host copy
    ctx.set_residency(1)
    assert np.array_equal(ctx.packed(k, 1)[0], ref.packed(k, 1)[0])


def test_ray_form_and_batch_exclusion():
    sc, cams, mlp = _scene()
    ctx = cow.Context(sc, "bf16")
    ids = list(range(4))
    o, d = synth.random_rays(4096, 3, sc.box_lo, sc.box_hi, device="cuda")
    want = ctx.render_rays(o, d, ids, mlp)[0]
    batch = cow.Batch(ctx, 2, 64)
    with pytest.raises(cow.CowError):
        ctx.set_residency(1 << 30)  # a live batch needs every block resident
    batch.close()
    ctx.set_residency(sum(ctx.block_bytes(i) for i in ids))
    got = ctx.render_rays(o, d, ids, mlp)[0]
    ctx.sync_check()
    assert torch.equal(got, want)
    with pytest.raises(cow.CowError):
        cow.Batch(ctx, 2, 64)
