"""Element-by-element comparison of a GPU gradient with the oracle's FP64
gradient at the differentiation form's tolerance (relative error <= 1e-3).

A norm alone would let a few wrong entries of a large grid hide inside it,
so a tensor passes only when all three hold:
  * relative L2 error <= rel;
  * every entry: |g - r| <= rel * max|r| (the tensor's scale);
  * every entry with |r| >= floor * max|r|: |g - r| <= rel * |r|."""
import numpy as np


def grad_errors(g, r, floor=0.1):
    """(relative L2, worst |g - r| / max|r|, worst |g - r| / |r| over the
    entries above floor * max|r|)."""
    g = np.asarray(g.detach().cpu().numpy() if hasattr(g, "detach") else g, np.float64).ravel()
    r = np.asarray(r.detach().cpu().numpy() if hasattr(r, "detach") else r, np.float64).ravel()
    scale = float(np.abs(r).max()) if r.size else 0.0
    if scale == 0.0:
        z = float(np.abs(g).max()) if g.size else 0.0
        return z, z, z
    e = np.abs(g - r)
    l2 = float(np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-300))
    big = np.abs(r) >= floor * scale
    rel_big = float((e[big] / np.abs(r[big])).max()) if big.any() else 0.0
    return l2, float(e.max()) / scale, rel_big


def assert_grad(g, r, what="", rel=1e-3, floor=0.1):
    l2, worst, worst_big = grad_errors(g, r, floor)
    assert l2 <= rel and worst <= rel and worst_big <= rel, (
        f"{what}: relative L2 {l2:.3g}, max entry error / max|ref| {worst:.3g}, "
        f"max relative error on entries >= {floor} max|ref| {worst_big:.3g} (bound {rel})")
