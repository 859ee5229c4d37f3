"""Oracle of off-grid receiver sampling pinned to closed forms: multilinear interpolation
reproduces fields linear in each logical index exactly, weights are a partition of unity,
receivers on nodes reduce to the on-grid selection, and the interpolated Jacobian pairs
with its transpose."""
import numpy as np

from paper_2609_14982_b300 import workloads as W


def test_interp_closed_forms(oracle_mod):
    n = (7, 6, 5)
    g = W.Grid(3, n, (1.0, 1.0, 1.0), np.zeros((int(np.prod(n)), 3)))
    rng = np.random.default_rng(2)
    f = rng.uniform(0, 1, (50, 3)) * (np.array(n) - 1)
    f[0] = [6.0, 5.0, 4.0]                       # the far corner (clamped base)
    P = oracle_mod.receiver_interp(g, f)
    assert np.allclose(P @ np.ones(P.shape[1]), 1.0, rtol=0, atol=1e-15)
    i, j, k = np.meshgrid(*[np.arange(m) for m in n], indexing="ij")
    for field, exact in (((1.5 * i - 2.0 * j + 0.25 * k).ravel(), 1.5 * f[:, 0] - 2.0 * f[:, 1] + 0.25 * f[:, 2]),
                         ((i * j * k).ravel().astype(float), f[:, 0] * f[:, 1] * f[:, 2])):
        assert np.allclose(P @ field, exact, rtol=0, atol=1e-12)
    on = np.array([[2, 3, 1], [0, 0, 0], [6, 5, 4]], dtype=float)
    Pn = oracle_mod.receiver_interp(g, on).toarray()
    sel = np.zeros_like(Pn)
    for r, (a, b, c) in enumerate(on.astype(int)):
        sel[r, g.index(a, b, c)] = 1.0
    assert np.array_equal(Pn, sel)


def test_interp_jacobian_pairing(oracle_mod):
    g = W.graph_grid((9, 9, 5), 300.0)
    _, G, _ = oracle_mod.metric(g)
    srcs = (W.quarter_source(g), W.centre_source(g))
    st = [W.curved_state(g, k, 0.05) for k in srcs]
    s = st[0].s
    tans = [oracle_mod.build_tangent(g, G, x.T, s, x.src) for x in st]
    rng = np.random.default_rng(6)
    Ps = [oracle_mod.receiver_interp(g, np.c_[rng.uniform(0, 8, (12, 2)), np.zeros(12)]) for _ in srcs]
    p = rng.standard_normal((g.N, 3))
    y = rng.standard_normal((2, 12, 3))
    l1 = float(np.sum(oracle_mod.J_interp(tans, s, Ps, p) * y))
    l2 = float(np.sum(p * oracle_mod.JT_interp(tans, s, Ps, y)))
    assert abs(l1 - l2) <= 1e-12 * max(abs(l1), abs(l2))
