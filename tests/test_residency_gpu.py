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


def test_ray_form_under_budget():
    sc, cams, mlp = _scene()
    ctx = cow.Context(sc, "bf16")
    ids = list(range(4))
    o, d = synth.random_rays(4096, 3, sc.box_lo, sc.box_hi, device="cuda")
    want = ctx.render_rays(o, d, ids, mlp)[0]
    ctx.set_residency(sum(ctx.block_bytes(i) for i in ids))
    got = ctx.render_rays(o, d, ids, mlp)[0]
    ctx.sync_check()
    assert torch.equal(got, want)


def _runs(bb, ids, budget):
    """The batch's cut of its views, in order, into runs whose distinct
    blocks fit the budget together."""
    runs, run, first = [], set(), 0
    for v, iv in enumerate(ids):
        own = set(int(i) for i in iv)
        add = sum(bb[i] for i in own - run)
        if v > first and sum(bb[i] for i in run) + add > budget:
            runs.append(run)
            run, first = set(), v
        run |= own
    runs.append(run)
    return runs


def _lru_uploads(bb, runs, budget, resident=()):
    """Bytes loaded when each run's blocks are made resident in turn by the
    context's rule: unload the least recently used blocks the run does not
    use (ties: lowest index) until the missing ones fit, then load them."""
    res, last, clock, up = set(resident), {}, 0, 0
    for run in runs:
        clock += 1
        for i in run:
            last[i] = clock
        missing = sum(bb[i] for i in run if i not in res)
        cur = sum(bb[i] for i in res)
        while cur + missing > budget:
            victim = min((i for i in res if i not in run), key=lambda i: (last.get(i, 0), i))
            res.remove(victim)
            cur -= bb[victim]
        for i in sorted(run):
            if i not in res:
                res.add(i)
                up += bb[i]
    return up, res


@pytest.mark.parametrize("run_frac", [1.0, 0.5])
def test_batch_under_budget_equals_all_resident(run_frac):
    """The batched form under a residency budget: the views run in groups
    whose blocks fit together in the run fraction of the budget, the pixels
    equal the all-resident batch's bit for bit, the loads equal a
    re-statement of the rule, the budget holds, and leaving the budget serves
    the whole batch in one launch again."""
    sc, cams, mlp = _scene()
    ref = cow.Context(sc, "bf16")
    ctx = cow.Context(sc, "bf16")
    ids = [ref.select_lod(c, sc.lod_thresh) for c in cams]
    mlp_d = torch.from_numpy(mlp).cuda()
    n_ids = sum(len(i) for i in ids)

    def outs(n):
        return (torch.empty((n, 3), device="cuda"), torch.empty((n, 8), device="cuda"),
                torch.empty(n, dtype=torch.int32, device="cuda"))

    rb = cow.Batch(ref, len(cams), n_ids)
    npix = rb.set_views(cams, ids)
    want = outs(npix)
    rb.render(mlp_d, *want)
    ref.sync_check()
    bb = [ctx.block_bytes(i) for i in range(len(sc.blocks))]
    need = [sum(bb[i] for i in set(v.tolist())) for v in ids]
    budget = int(1.25 * max(need))
    batch = cow.Batch(ctx, len(cams), n_ids)  # created before the budget is set
    batch.set_run_fraction(run_frac)
    assert batch.set_views(cams, ids) == npix
    got = outs(npix)
    batch.render(mlp_d, *got, graph=True)
    assert batch.last_groups() == 1
    ctx.set_residency(budget)
    r0 = ctx.residency()
    cap = int(budget * run_frac)
    runs = _runs(bb, ids, cap)
    runs_back = _runs(bb, ids[::-1], cap)  # the second render walks the views last to first
    assert len(runs) > 2
    for step in range(2):  # the second render starts from what the first left resident
        for t in got:
            t.zero_()
        before = ctx.residency()
        batch.render(mlp_d, *got, graph=True)
        ctx.sync_check()
        assert batch.last_groups() == len(runs if step == 0 else runs_back)
        after = ctx.residency()
        assert after["resident_bytes"] <= budget
        for g, w in zip(got, want):
            assert torch.equal(g, w)
        if step == 0:
            up, left = _lru_uploads(bb, runs, budget)
            assert after["upload_bytes"] - r0["upload_bytes"] == up
            assert after["resident_bytes"] == sum(bb[i] for i in left)
        else:  # it begins with the last run's blocks, still resident: fewer loads than a cold walk
            up_back, _ = _lru_uploads(bb, runs_back, budget)
            assert 0 < after["upload_bytes"] - before["upload_bytes"] < up_back
    # back to all resident: new block records, one launch (graph replay)
    ctx.set_residency(0)
    for t in got:
        t.zero_()
    batch.render(mlp_d, *got, graph=True)
    ctx.sync_check()
    assert batch.last_groups() == 1
    for g, w in zip(got, want):
        assert torch.equal(g, w)
    # a view whose blocks alone exceed the budget
    ctx.set_residency(max(need) - 1)
    with pytest.raises(cow.CowError) as e:
        batch.render(mlp_d, got[0])
    assert e.value.status == 3  # OOM
    assert ctx.residency()["resident_bytes"] <= max(need) - 1
    batch.close()
    rb.close()
