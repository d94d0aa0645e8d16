"""Failure detection without a GPU fault: the kernels' own checks end in an
error status that the host reads, and the context stays usable.

* Bounded waits: the kernels that stage a view's block records with a TMA
  bulk copy wait for it on an mbarrier with an iteration limit.  The test
  hook COW_TEST_SKIP_RECORD_COPY leaves the copy unissued (the barrier's
  phase never completes, nothing is in flight) and a short poll limit makes
  the wait run out: cow_sync_check returns COW_ERR_TIMEOUT.
* Range check: a (ray, block) pair whose candidate lattice range exceeds
  2^22 indices is clamped and recorded: cow_sync_check returns
  COW_ERR_DEVICE_ASSERT.  The input is legitimate: a block 1e-4 wide and
  1000 tall, looked at straight down (a lattice step of 5e-5 along a
  1000-long ray)."""
import numpy as np
import pytest
import torch

from paper_2312_16457_gb300 import cow, synth

pytestmark = pytest.mark.gpu

TIMEOUT, DEVICE_ASSERT = 5, 6


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2312_16457_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def _status(fn):
    with pytest.raises(cow.CowError) as e:
        fn()
    return e.value.status


def _small():
    sc = synth.city_scene(21, 2, 2.0, [(12, 16)])
    cam = synth.camera((-2.5, -3.0, 2.2), (0.3, 0.4, -0.8), 40, 24, 60.0)
    return sc, cam, synth.mlp_weights(3)


@pytest.mark.parametrize("schedule", ["thread", "warp"])
def test_view_record_wait_times_out(schedule):
    sc, cam, mlp = _small()
    ctx = cow.Context(sc, "bf16")
    ctx.set_schedule(schedule)
    ids = [ctx.sort_blocks(cam, list(range(4)))]
    ref = ctx.render([cam], ids, mlp, nsamp=True)
    ctx.sync_check()
    ctx.set_test_hooks(skip_record_copy=True, wait_polls=1024)
    ctx.render([cam], ids, mlp)
    assert _status(ctx.sync_check) == TIMEOUT
    ctx.set_test_hooks()  # the context stays usable
    again = ctx.render([cam], ids, mlp, nsamp=True)
    ctx.sync_check()
    for x, y in zip(ref, again):
        assert torch.equal(x, y)
    ctx.close()


def test_batch_record_wait_times_out():
    """The batched form stages records with a bulk copy when its record mode
    is "shared" (otherwise runs take their records in the parameter buffer
    and nothing waits), here under a residency budget as well."""
    sc, cam, mlp = _small()
    ctx = cow.Context(sc, "bf16")
    cams = [cam, synth.camera((2.0, 2.5, 1.5), (-0.2, -0.1, -0.9), 32, 32, 60.0)]
    ids = [ctx.sort_blocks(c, list(range(4))) for c in cams]
    mlp_d = torch.from_numpy(mlp).cuda()
    batch = cow.Batch(ctx, 2, 8)
    batch.set_records("shared")
    npix = batch.set_views(cams, ids)
    ref = torch.empty((npix, 3), device="cuda")
    batch.render(mlp_d, ref)
    ctx.sync_check()
    ctx.set_residency(sum(ctx.block_bytes(i) for i in range(4)))
    out = torch.full((npix, 3), -1.0, device="cuda")
    ctx.set_test_hooks(skip_record_copy=True, wait_polls=1024)
    batch.render(mlp_d, out)
    assert _status(ctx.sync_check) == TIMEOUT
    assert bool((out == -1.0).all())  # the CTAs left without writing pixels
    ctx.set_test_hooks()
    batch.render(mlp_d, out)
    ctx.sync_check()
    assert torch.equal(out, ref)
    ctx.set_residency(0)
    batch.close()
    ctx.close()


def test_context_freed_before_its_batch():
    """A batch outliving its context (garbage collection can free them in
    either order) is detached: its calls fail cleanly and freeing it works."""
    sc, cam, mlp = _small()
    ctx = cow.Context(sc, "bf16")
    batch = cow.Batch(ctx, 1, 8)
    npix = batch.set_views([cam], [ctx.sort_blocks(cam, list(range(4)))])
    ctx.close()
    with pytest.raises(cow.CowError, match="freed"):
        batch.render(torch.from_numpy(mlp).cuda(), torch.empty((npix, 3), device="cuda"))
    batch.close()
    # the runtime's error state is clean: a new context loads
    ctx2 = cow.Context(sc, "bf16")
    ctx2.sync_check()
    ctx2.close()


def test_default_schedule_has_no_wait():
    """The default schedule takes its records in the parameter buffer: the
    hook changes nothing there."""
    sc, cam, mlp = _small()
    ctx = cow.Context(sc, "bf16")
    ids = [ctx.sort_blocks(cam, list(range(4)))]
    ref = ctx.render([cam], ids, mlp)[0]
    ctx.set_test_hooks(skip_record_copy=True, wait_polls=1024)
    got = ctx.render([cam], ids, mlp)[0]
    ctx.sync_check()
    assert torch.equal(ref, got)
    ctx.close()


def test_range_check_reports_device_assert():
    R, P = 2, 2
    g = torch.zeros(R, R, R, 8)
    g[..., 0] = np.log(1e-4)  # empty: the clamped range is crossed in one jump
    pl = [torch.zeros(P, P, 8) for _ in range(3)]
    blk = synth.Block((0.0, 0.0, -500.0), (1e-4, 1e-4, 500.0), R, P, grid=g, planes=pl)
    sc = synth.Scene([blk], blk.lo, blk.hi)
    ctx = cow.Context(sc, "fp32")
    c2w = np.array([[1.0, 0, 0, 5e-5], [0, 1.0, 0, 5e-5], [0, 0, 1.0, 600.0]])  # looking down -z
    cam = synth.Camera(c2w, 1, 1, 1e-3)
    mlp = synth.mlp_weights(3)
    ctx.render([cam], [[0]], mlp)
    assert _status(ctx.sync_check) == DEVICE_ASSERT
    # a ray that stays within the bound leaves the error word clear
    cam2 = synth.Camera(np.array([[1.0, 0, 0, 5e-5], [0, 0, -1.0, -1.0], [0, 1.0, 0, 0.0]]), 1, 1, 1e-3)  # along +y
    ctx.render([cam2], [[0]], mlp)
    ctx.sync_check()
    ctx.close()
