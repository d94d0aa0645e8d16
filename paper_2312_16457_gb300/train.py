"""Differentiation form: a torch.autograd.Function over libcow's ray-batch
render and its backward kernels, and a fitter that optimises block features
and the deferred MLP with libcow's Adam kernel.

Gradients come from cow_render_backward (re-marching each ray from its saved
totals); the optimiser step, the loss gradient and the re-packing of the
updated features run in libcow kernels as well.  Occupancy stays as loaded.
"""
from __future__ import annotations

from typing import List, Sequence

import torch

from . import cow


class RenderRays(torch.autograd.Function):
    """rgb = render(o, d; features, mlp).  Inputs: the context, block ids, the
    MLP (499) and the flat feature parameters [grid_0, xy_0, xz_0, yz_0, grid_1,
    ...] of every block of the context (FP32 device tensors)."""

    @staticmethod
    def forward(fctx, cctx: cow.Context, ids: Sequence[int], o, d, ert_eps: float, mlp, *params):
        nb = cctx.n_blocks
        assert len(params) == 4 * nb
        for i in range(nb):
            cctx.update_features(i, params[4 * i], params[4 * i + 1:4 * i + 4])
        rgb, aux, _ = cctx.render_rays(o, d, ids, mlp.detach(), ert_eps=ert_eps)
        fctx.save_for_backward(o, d, mlp, aux)
        fctx.cctx, fctx.ids, fctx.ert = cctx, list(ids), ert_eps
        fctx.shapes = [p.shape for p in params]
        return rgb

    @staticmethod
    def backward(fctx, grad_rgb):
        o, d, mlp, aux = fctx.saved_tensors
        cctx = fctx.cctx
        nb = cctx.n_blocks
        grads = [torch.zeros(s, dtype=torch.float32, device=o.device) for s in fctx.shapes]
        gm = torch.zeros(499, dtype=torch.float32, device=o.device)
        cctx.render_backward(o, d, fctx.ids, mlp.detach().contiguous(), aux, grad_rgb.contiguous().float(),
                             [grads[4 * i] for i in range(nb)], [grads[4 * i + 1:4 * i + 4] for i in range(nb)], gm,
                             ert_eps=fctx.ert)
        return (None, None, None, None, None, gm, *grads)


def render_rays(cctx: cow.Context, ids, o, d, mlp, params: List[torch.Tensor], ert_eps: float = 0.0):
    return RenderRays.apply(cctx, ids, o, d, ert_eps, mlp, *params)


class Fitter:
    """Fit block features and the deferred MLP to target colours of a ray
    batch: forward, MSE gradient, backward, Adam, re-pack -- all in libcow."""

    def __init__(self, scene, mlp, lr_feat=1e-2, lr_mlp=1e-3, device="cuda", lambda_sparsity=0.0,
                 lambda_opacity=0.0, n_sparsity_points=1 << 14, seed=0, block_mlps=None, n_freq=0,
                 storage="fp32"):
        """lambda_sparsity / lambda_opacity weight the regularisers of Eq. 7
        (mean alpha at n_sparsity_points uniform points of the scene box,
        redrawn every step) and Eq. 8 (entropy of block opacities of the
        step's rays); the paper trains with 0.05 and 0.001.  block_mlps
        ([n_blocks, block_mlp_nparam(n_freq)]) fits one MLP per block,
        blended by Eq. 5, instead of the global `mlp` (which may be None);
        that form has no early termination.  storage: the packed copies the
        forward and backward read ("fp32", or "bf16" / "fp16" re-packed from
        the FP32 parameters after every Adam step: FP32 masters, FP32
        gradients and optimiser, reduced-precision renders)."""
        self.ctx = cow.Context(scene, storage)
        self.box_lo = torch.tensor(scene.box_lo, dtype=torch.float32, device=device)
        self.box_hi = torch.tensor(scene.box_hi, dtype=torch.float32, device=device)
        self.lambda_sparsity, self.lambda_opacity = float(lambda_sparsity), float(lambda_opacity)
        self.n_sparsity_points = int(n_sparsity_points)
        self.gen = torch.Generator(device=device)
        self.gen.manual_seed(seed)
        self.reg_loss = None
        self.ids = list(range(len(scene.blocks)))
        self.params = []
        for b in scene.blocks:
            self.params += [b.grid.to(device).float().contiguous()] + [p.to(device).float().contiguous() for p in b.planes]
        self.n_freq = int(n_freq)
        if block_mlps is not None:
            self.block_mlps = torch.as_tensor(block_mlps, dtype=torch.float32, device=device).contiguous()
            self.ctx.set_block_mlps(self.block_mlps, self.n_freq)
            self.mlp = None
            mw = self.block_mlps
        else:
            self.block_mlps = None
            self.mlp = torch.as_tensor(mlp, dtype=torch.float32, device=device).contiguous()
            mw = self.mlp
        self.m = [torch.zeros_like(p) for p in self.params] + [torch.zeros_like(mw)]
        self.v = [torch.zeros_like(p) for p in self.params] + [torch.zeros_like(mw)]
        self.lr_feat, self.lr_mlp = lr_feat, lr_mlp
        self.t = 0

    def step(self, o, d, target, ert_eps: float = 0.0):
        """One optimisation step; returns the colour loss (device tensor)
        before it (the weighted regularisers are in self.reg_loss)."""
        nb = len(self.ids)
        block_T = None
        per_block = self.block_mlps is not None
        if per_block:
            if ert_eps != 0.0:
                raise ValueError("the per-block MLP form fits without early termination")
            # the forward keeps every (ray, block) state, so the backward marches once
            rgb, bm_state = self.ctx.render_rays_block_state(o, d, self.ids)
        elif self.lambda_opacity > 0.0 and ert_eps == 0.0:
            # the forward also keeps every block's transmittance for the opacity term
            rgb, aux, block_T = self.ctx.render_rays_block_t(o, d, self.ids, self.mlp)
        else:
            rgb, aux, _ = self.ctx.render_rays(o, d, self.ids, self.mlp, ert_eps=ert_eps)
        g, loss = cow.mse_grad(rgb, target)
        grads = [torch.zeros_like(p) for p in self.params]
        gtab = ([grads[4 * i] for i in range(nb)], [grads[4 * i + 1:4 * i + 4] for i in range(nb)])
        if per_block:
            gm = torch.zeros_like(self.block_mlps)
            self.ctx.render_backward_block_mlps_state(o, d, self.ids, bm_state, g, gtab[0], gtab[1], gm)
        else:
            gm = torch.zeros_like(self.mlp)
            self.ctx.render_backward(o, d, self.ids, self.mlp, aux, g, gtab[0], gtab[1], gm, ert_eps=ert_eps)
        if self.lambda_sparsity > 0.0 or self.lambda_opacity > 0.0:
            self.reg_loss = torch.zeros(1, dtype=torch.float32, device=o.device)
            if self.lambda_sparsity > 0.0:
                u = torch.rand((self.n_sparsity_points, 3), generator=self.gen, device=o.device)
                pts = self.box_lo + u * (self.box_hi - self.box_lo)
                self.ctx.sparsity_loss(pts, self.ids, self.lambda_sparsity, loss=self.reg_loss, grads=gtab)
            if self.lambda_opacity > 0.0:
                self.ctx.opacity_loss(o, d, self.ids, self.lambda_opacity, loss=self.reg_loss, grads=gtab,
                                      block_T=block_T)
        self.t += 1
        for k, p in enumerate(self.params):
            cow.adam_step(p, grads[k], self.m[k], self.v[k], self.lr_feat, self.t)
        if per_block:
            cow.adam_step(self.block_mlps, gm, self.m[-1], self.v[-1], self.lr_mlp, self.t)
            self.ctx.set_block_mlps(self.block_mlps, self.n_freq)
        else:
            cow.adam_step(self.mlp, gm, self.m[-1], self.v[-1], self.lr_mlp, self.t)
        for i in range(nb):
            self.ctx.update_features(i, self.params[4 * i], self.params[4 * i + 1:4 * i + 4])
        return loss

    def state_dict(self) -> dict:
        """Everything a resumed fit needs: the FP32 parameters, the MLP (or
        per-block MLPs), Adam's moments and step count, the learning rates."""
        return {"params": [p.detach().cpu() for p in self.params],
                "mlp": None if self.mlp is None else self.mlp.detach().cpu(),
                "block_mlps": None if self.block_mlps is None else self.block_mlps.detach().cpu(),
                "n_freq": self.n_freq, "m": [x.detach().cpu() for x in self.m], "v": [x.detach().cpu() for x in self.v],
                "t": self.t, "lr_feat": self.lr_feat, "lr_mlp": self.lr_mlp, "rng": self.gen.get_state().cpu()}

    def save(self, path: str):
        """Checkpoint of the fit (torch.save of state_dict())."""
        torch.save(self.state_dict(), path)

    def load(self, path_or_state):
        """Resume from save(): parameters and Adam state are restored and the
        context's packed features re-packed from the parameters."""
        st = torch.load(path_or_state, map_location="cpu") if isinstance(path_or_state, str) else path_or_state
        if len(st["params"]) != len(self.params) or (st["block_mlps"] is None) != (self.block_mlps is None):
            raise ValueError("checkpoint of a different fit")
        for p, q in zip(self.params, st["params"]):
            p.copy_(q.to(p.device))
        for x, q in zip(self.m, st["m"]):
            x.copy_(q.to(x.device))
        for x, q in zip(self.v, st["v"]):
            x.copy_(q.to(x.device))
        if self.block_mlps is not None:
            self.block_mlps.copy_(st["block_mlps"].to(self.block_mlps.device))
            self.ctx.set_block_mlps(self.block_mlps, self.n_freq)
        else:
            self.mlp.copy_(st["mlp"].to(self.mlp.device))
        self.t = int(st["t"])
        self.lr_feat, self.lr_mlp = st["lr_feat"], st["lr_mlp"]
        self.gen.set_state(st["rng"].to(self.gen.get_state().device))
        for i in range(len(self.ids)):
            self.ctx.update_features(i, self.params[4 * i], self.params[4 * i + 1:4 * i + 4])

    def render(self, o, d, ert_eps: float = 0.0):
        if self.block_mlps is not None:
            return self.ctx.render_rays(o, d, self.ids, None, aux=False, block_mlps=True)[0]
        return self.ctx.render_rays(o, d, self.ids, self.mlp, ert_eps=ert_eps, aux=False)[0]
