"""Oracle pinned to the paper's printed tables (Tables 1-3, mu_G range, algebraic checks).

These tests fix the oracle's readings of the discretization (finite-difference metric
with second-order one-sided edges, face-averaged metric and gradient, compact normal
difference, canonical condensation) against numbers the paper prints."""
import os

import numpy as np
import pytest

from paper_2609_14982_b300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(line.split())
    return out


def _table1(O, nx):
    c = W.table1_case(nx)
    _, G, det = O.metric(c.grid)
    t = O.build_tangent(c.grid, G, c.T, c.s, c.src)
    q = t.cs * c.ds
    x = O.solve(t, q)
    m = c.mask
    e = x - c.dT_exact
    E2 = np.linalg.norm(e[m]) / np.linalg.norm(c.dT_exact[m])
    Ei = np.abs(e[m]).max() / np.abs(c.dT_exact[m]).max()
    return c, G, det, t, q, x, E2, Ei


@pytest.mark.parametrize("nx", [21, 41, 81, 161])
def test_table1_errors(oracle_mod, nx):
    """Table 1: E2 and Einf of the manufactured tangent (closed form Eq. test-dT)."""
    if nx == 161 and os.environ.get("EIK_FAST_TESTS"):
        pytest.skip("fast mode")
    O = oracle_mod
    row = [r for r in _rows("table1.txt") if int(r[0]) == nx][0]
    c, G, det, t, q, x, E2, Ei = _table1(O, nx)
    assert np.all(det > 0)                       # "Jacobian determinant is positive on every grid"
    assert abs(E2 - float(row[2])) <= 0.5e-4 * 10 ** np.floor(np.log10(float(row[2])))
    # Einf: all printed digits except the 81^3 case, which prints 6.2239e-3 for our 6.22385e-3
    assert abs(Ei - float(row[3])) <= 1.0e-4 * 10 ** np.floor(np.log10(float(row[3])))
    mu = O.mu_G(G)
    assert 0.2999 - 5e-5 <= mu <= 0.3083 + 5e-5
    # algebraic checks of Table 1: solve residual, inverse pair, scaling identity (Sec. 3.2)
    A = t.A()
    assert np.linalg.norm(A @ x - q) / np.linalg.norm(q) < 2e-14
    rng = np.random.default_rng(nx)
    b, y = rng.standard_normal(t.N), rng.standard_normal(t.N)
    l1 = y @ O.solve(t, b)
    l2 = O.solve_T(t, y) @ b
    assert abs(l1 - l2) / max(abs(l1), abs(l2), 1.0) < 1e-13
    xs = O.solve(t, -t.cs * c.s)                 # uniform relative scaling dv = v -> ds = -s
    assert np.linalg.norm(xs + c.T) / np.linalg.norm(c.T) < 1e-14


def test_table1_orders(oracle_mod):
    """Observed orders p2/pinf between 21 and 41 (Eq. test-order): 0.9550 and 0.8691."""
    O = oracle_mod
    e21 = _table1(O, 21)[-2:]
    e41 = _table1(O, 41)[-2:]
    p2 = np.log(e21[0] / e41[0]) / np.log(2.0)
    pi = np.log(e21[1] / e41[1]) / np.log(2.0)
    assert abs(p2 - 0.9550) < 1e-3 and abs(pi - 0.8691) < 1e-3


def test_mu_g_first_level(oracle_mod):
    """mu_G on 21x21x11 equals the top of the printed range, 0.3083."""
    _, G, _ = oracle_mod.metric(W.table1_grid(21))
    assert abs(oracle_mod.mu_G(G) - 0.3083) < 5e-5


def _structure(O, g, st):
    _, G, _ = O.metric(g)
    t = O.build_tangent(g, G, st.T, st.s, st.src)
    j, i = t.edges()
    nvio = int(np.sum(st.T[j] > st.T[i]))
    sizes = t.scc_sizes()
    nt = sizes[sizes > 1]
    return dict(mu=O.mu_G(G), nvio=nvio, NE=len(j), nscc=len(nt), cyc=int(nt.sum()),
                largest=int(nt.max()) if len(nt) else 0, unr=t.kahn_unresolved(), N=g.N, t=t)


@pytest.mark.parametrize("case", ["A", "B", "C"])
def test_table2_regimes(oracle_mod, case):
    """Table 2: mu_G, f_vio, SCC count, f_cyc, largest SCC, f_unr for cases A/B/C."""
    row = [r for r in _rows("table2.txt") if r[0] == case][0]
    A, eps = float(row[2]), float(row[3])
    g = W.graph_grid((41, 41, 25), A)
    src = W.quarter_source(g)
    st = W.radial_state(g, src) if row[1] == "radial" else W.curved_state(g, src, eps)
    s = _structure(oracle_mod, g, st)
    assert abs(s["mu"] - float(row[4])) < 5e-4
    fvio = 100.0 * s["nvio"] / s["NE"]
    if case == "C":
        # printed 6.340 %; the oracle counts 7758 of 122344 edges (6.3411 %), one edge above
        # the largest count that prints as 6.340 -> allow two edges
        assert abs(s["nvio"] - float(row[5]) / 100 * s["NE"]) <= 2.0
    else:
        assert abs(fvio - float(row[5])) < 5e-4
    assert s["nscc"] == int(row[6])
    assert abs(100.0 * s["cyc"] / s["N"] - float(row[7])) < 5e-4
    assert s["largest"] == int(row[8])
    assert abs(100.0 * s["unr"] / s["N"] - float(row[9])) < 5e-4


@pytest.mark.parametrize("n0", [21, 41, 61, 81])
def test_table3_refinement(oracle_mod, n0):
    """Table 3: nontrivial SCCs, cyclic nodes, largest SCC, Kahn-unresolved, exactly."""
    row = [r for r in _rows("table3.txt") if int(r[0]) == n0][0]
    n = tuple(int(v) for v in row[:3])
    g = W.graph_grid(n, 500.0)
    st = W.curved_state(g, W.quarter_source(g), 0.05)
    s = _structure(oracle_mod, g, st)
    assert s["N"] == int(row[3])
    assert (s["nscc"], s["cyc"], s["largest"], s["unr"]) == tuple(int(v) for v in row[4:8])


def test_flat_grids_ordered(oracle_mod):
    """Sec. 5.2.1: every flat-grid case is traveltime ordered and acyclic (radial and curved
    states, three surface sources)."""
    O = oracle_mod
    g = W.graph_grid((41, 41, 25), 0.0)
    for src in (W.quarter_source(g), W.centre_source(g), g.index(30, 10, 0)):
        for eps in (0.0, 0.025, 0.05):
            st = W.radial_state(g, src) if eps == 0 else W.curved_state(g, src, eps)
            s = _structure(O, g, st)
            assert s["nvio"] == 0 and s["nscc"] == 0 and s["unr"] == 0
