"""Oracle pin of the block-parallel form (Eq. 12-13, App. A): every block
rendered alone gives its partial (C_d^k, F^k, T^k); folding those near to
far with the "over" (C, F, T) <- (C + T C^k, F + T F^k, T T^k) reproduces the
oracle's block-sequential render of the same rays, and the fold is
associative (any bracketing of the blocks gives the same result)."""
import numpy as np

from paper_2312_16457_gb300 import synth


def _over(a, b):
    """(C, F, T) of a in front of b: 8-vectors C_d (3), F (4), T."""
    out = np.empty(8)
    out[:7] = a[:7] + a[7] * b[:7]
    out[7] = a[7] * b[7]
    return out


def test_over_of_single_block_partials_is_the_block_sequential_render(orc):
    sc = synth.city_scene(23, 2, 2.0, [(10, 16)])
    osc = orc.OracleScene(sc)
    o, d = synth.random_rays(96, 5, sc.box_lo, sc.box_hi)
    o, d = o.numpy(), d.numpy()
    ids = [0, 1, 2, 3]
    _, full, ns = orc.render_rays(osc, ids, o, d)
    parts = [orc.render_rays(osc, [k], o, d)[1] for k in ids]
    crossing = 0
    for r in range(len(o)):
        order = orc.sort_ids_for_ray(osc, ids, o[r])
        acc = np.array([0.0] * 7 + [1.0])
        for k in order:
            acc = _over(acc, parts[k][r])
        np.testing.assert_allclose(acc, full[r], rtol=0, atol=1e-12)
        crossing += sum(parts[k][r][7] < 1.0 for k in ids) > 1
    assert crossing >= 10 and ns.sum() > 0  # rays through several occupied blocks


def test_over_is_associative():
    rng = np.random.default_rng(3)
    for _ in range(20):
        p = [np.concatenate([rng.uniform(0, 1, 7), rng.uniform(0.05, 1, 1)]) for _ in range(6)]
        left = p[0]
        for q in p[1:]:
            left = _over(left, q)
        right = p[-1]
        for q in reversed(p[:-1]):
            right = _over(q, right)
        tree = _over(_over(_over(p[0], p[1]), _over(p[2], p[3])), _over(p[4], p[5]))
        np.testing.assert_allclose(left, right, rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(left, tree, rtol=1e-14, atol=1e-14)
