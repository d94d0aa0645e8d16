"""The element-by-element gradient comparison itself (CPU): a few wrong
entries of a large tensor that a relative-L2 bound alone lets through must
fail it."""
import numpy as np

from gradcheck import grad_errors


def test_one_wrong_entry_fails_entrywise_but_not_in_norm():
    rng = np.random.default_rng(0)
    r = rng.normal(size=200000)
    g = r * (1.0 + 1e-7 * rng.normal(size=r.size))
    l2, worst, worst_big = grad_errors(g, r)
    assert l2 <= 1e-3 and worst <= 1e-3 and worst_big <= 1e-3
    k = int(np.argmax(np.abs(r)))
    g2 = g.copy()
    g2[k] *= 1.05  # 5 % off on the largest entry
    l2, worst, worst_big = grad_errors(g2, r)
    assert l2 <= 1e-3  # the norm hides it
    assert worst > 1e-3 and worst_big > 1e-3


def test_relative_bound_on_large_entries():
    r = np.array([100.0, 20.0, 1e-6])
    g = r + np.array([0.0, 0.05, 0.0])  # 0.25 % of a large entry, 5e-4 of the scale
    _, worst, worst_big = grad_errors(g, r)
    assert worst <= 1e-3 < worst_big
