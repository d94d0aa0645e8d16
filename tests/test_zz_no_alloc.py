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


def _rel(a, b):
    a = a.double().cpu().numpy().ravel()
    b = b.double().cpu().numpy().ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _zeros(sc):
    gg = [torch.zeros(b.grid.shape, device="cuda") for b in sc.blocks]
    gp = [[torch.zeros(p.shape, device="cuda") for p in b.planes] for b in sc.blocks]
    return gg, gp, torch.zeros(499, device="cuda")


def test_noalloc_backward_matches_regular_backward():
    sc = synth.city_scene(17, 2, 2.0, [(16, 40)])
    n = 6000
    o, d = synth.random_rays(n, 7, sc.box_lo, sc.box_hi)
    o, d = o.cuda(), d.cuda()
    ids = [0, 1, 2, 3]
    mlp = torch.from_numpy(synth.mlp_weights(8)).cuda()
    g = torch.from_numpy(np.random.default_rng(4).normal(size=(n, 3)).astype(np.float32)).cuda()
    ctx = cow.Context(sc, "fp32")
    _, aux, _ = ctx.render_rays(o, d, ids, mlp)
    ref_g, ref_p, ref_m = _zeros(sc)
    ctx.render_backward(o, d, ids, mlp, aux, g, ref_g, ref_p, ref_m)
    ctx.sync_check()
    for call in range(2):  # two calls in a row share the static scratch
        gg, gp, gm = _zeros(sc)
        ctx.render_backward(o, d, ids, mlp, aux, g, gg, gp, gm, noalloc=True)
        ctx.sync_check()
        assert _rel(gm, ref_m) <= 1e-5, call
        for b in range(4):
            assert _rel(gg[b], ref_g[b]) <= 1e-5, (call, b)
            for k in range(3):
                assert _rel(gp[b][k], ref_p[b][k]) <= 1e-5, (call, b, k)
        assert float(gm.abs().max()) > 0.0


def test_noalloc_backward_rejects_oversize():
    sc = synth.city_scene(17, 2, 2.0, [(8, 16)])
    n = 65537
    o, d = synth.random_rays(n, 7, sc.box_lo, sc.box_hi)
    o, d = o.cuda(), d.cuda()
    mlp = torch.from_numpy(synth.mlp_weights(8)).cuda()
    ctx = cow.Context(sc, "fp32")
    _, aux, _ = ctx.render_rays(o, d, [0, 1, 2, 3], mlp)
    gg, gp, gm = _zeros(sc)
    with pytest.raises(cow.CowError, match="65536"):
        ctx.render_backward(o, d, [0, 1, 2, 3], mlp, aux, torch.zeros(n, 3, device="cuda"), gg, gp, gm, noalloc=True)
