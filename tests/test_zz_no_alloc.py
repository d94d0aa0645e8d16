"""The allocation-free backward (cow_render_backward_noalloc) against the
regular backward (cow_render_backward), through the C ABI.

The variant exists for callers that cannot allocate device memory once they
run (a fixed device-memory budget, or a loop that must not pay for
cudaMalloc / cudaFree); it keeps its scratch in a static device array of the
library.  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes on its own."""
import numpy as np
import pytest
import torch

from paper_2312_16457_gb300 import cow, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2312_16457_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def _close(a, b, rel=1e-5):
    """Entry by entry: |a - b| <= rel * max|b| (both runs scatter with float
    atomics, so the summation order differs), plus relative L2 <= rel."""
    a = a.double().cpu().numpy().ravel()
    b = b.double().cpu().numpy().ravel()
    scale = max(float(np.abs(b).max()), 1e-30)
    worst = float(np.abs(a - b).max()) / scale
    l2 = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
    return worst <= rel and l2 <= rel, (worst, l2)


def _zeros(sc):
    gg = [torch.zeros(b.grid.shape, device="cuda") for b in sc.blocks]
    gp = [[torch.zeros(p.shape, device="cuda") for p in b.planes] for b in sc.blocks]
    return gg, gp, torch.zeros(499, device="cuda")


def _setup(n, seed=7, res=(16, 40)):
    sc = synth.city_scene(17, 2, 2.0, [res])
    o, d = synth.random_rays(n, seed, sc.box_lo, sc.box_hi)
    o, d = o.cuda(), d.cuda()
    mlp = torch.from_numpy(synth.mlp_weights(8)).cuda()
    g = torch.from_numpy(np.random.default_rng(4).normal(size=(n, 3)).astype(np.float32)).cuda()
    return sc, o, d, mlp, g


def _check_against_regular(n):
    sc, o, d, mlp, g = _setup(n)
    ids = [0, 1, 2, 3]
    ctx = cow.Context(sc, "fp32")
    _, aux, _ = ctx.render_rays(o, d, ids, mlp)
    ref_g, ref_p, ref_m = _zeros(sc)
    ctx.render_backward(o, d, ids, mlp, aux, g, ref_g, ref_p, ref_m)
    ctx.sync_check()
    for call in range(2):  # two calls in a row share the static scratch
        gg, gp, gm = _zeros(sc)
        ctx.render_backward(o, d, ids, mlp, aux, g, gg, gp, gm, noalloc=True)
        ctx.sync_check()
        ok, why = _close(gm, ref_m)
        assert ok, (call, why)
        for b in range(4):
            ok, why = _close(gg[b], ref_g[b])
            assert ok, (call, b, why)
            for k in range(3):
                ok, why = _close(gp[b][k], ref_p[b][k])
                assert ok, (call, b, k, why)
        assert float(gm.abs().max()) > 0.0
    ctx.close()


def test_noalloc_backward_matches_regular_backward():
    _check_against_regular(6000)


def test_noalloc_backward_at_its_ray_limit():
    """Exactly 65536 rays, the largest call the static scratch holds."""
    _check_against_regular(65536)


def test_noalloc_backward_allocates_nothing():
    """A context that never ran the regular backward (so it holds no backward
    scratch): after one warm-up call (the first call on a device looks the
    static array up, and lazy module loading may map it), further calls
    leave the device's free memory unchanged."""
    sc, o, d, mlp, g = _setup(4096)
    ids = [0, 1, 2, 3]
    ctx = cow.Context(sc, "fp32")
    _, aux, _ = ctx.render_rays(o, d, ids, mlp)
    gg, gp, gm = _zeros(sc)
    ctx.render_backward(o, d, ids, mlp, aux, g, gg, gp, gm, noalloc=True)
    ctx.sync_check()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        ctx.render_backward(o, d, ids, mlp, aux, g, gg, gp, gm, noalloc=True)
    ctx.sync_check()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ctx.close()


def test_noalloc_backward_rejects_oversize():
    sc, o, d, mlp, _ = _setup(65537, res=(8, 16))
    ctx = cow.Context(sc, "fp32")
    _, aux, _ = ctx.render_rays(o, d, [0, 1, 2, 3], mlp)
    gg, gp, gm = _zeros(sc)
    with pytest.raises(cow.CowError, match="65536"):
        ctx.render_backward(o, d, [0, 1, 2, 3], mlp, aux, torch.zeros(65537, 3, device="cuda"), gg, gp, gm,
                            noalloc=True)
    ctx.close()


def test_noalloc_backward_rejects_more_than_1024_blocks():
    """A context of 33 x 33 tiny blocks: the call is refused on the host
    before any device work (its pointer table holds 1024 blocks)."""
    sc = synth.city_scene(5, 33, 0.5, [(2, 2)])
    assert len(sc.blocks) > 1024
    ctx = cow.Context(sc, "fp32")
    o = torch.zeros(8, 3, device="cuda")
    d = torch.zeros(8, 3, device="cuda")
    d[:, 2] = -1.0
    mlp = torch.from_numpy(synth.mlp_weights(8)).cuda()
    aux = torch.zeros(8, 8, device="cuda")
    gm = torch.zeros(499, device="cuda")
    nb = len(sc.blocks)
    with pytest.raises(cow.CowError, match="1024"):
        ctx.render_backward(o, d, [0], mlp, aux, torch.zeros(8, 3, device="cuda"), [None] * nb, [None] * nb, gm,
                            noalloc=True)
    ctx.close()


def test_noalloc_backward_rejects_unloaded_block():
    """Under a residency budget the variant loads nothing: a block that is
    not on the device is refused (the regular backward would load it)."""
    sc, o, d, mlp, g = _setup(512, res=(8, 16))
    ctx = cow.Context(sc, "fp32")
    _, aux, _ = ctx.render_rays(o, d, [0, 1, 2, 3], mlp)
    ctx.set_residency(sum(ctx.block_bytes(i) for i in range(4)))  # entering a budget unloads every block
    gg, gp, gm = _zeros(sc)
    with pytest.raises(cow.CowError, match="unloaded"):
        ctx.render_backward(o, d, [0, 1, 2, 3], mlp, aux, g, gg, gp, gm, noalloc=True)
    ctx.set_residency(0)
    ctx.close()
