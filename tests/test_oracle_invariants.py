"""Oracle pinned to mathematics other than itself: brute-force dense solves, a library SCC
routine, Props. 1-3, the M-matrix theorem, the adjoint pairing, the scaling identity and
the constant-gradient closed form."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import breadth_first_order, connected_components

from paper_2609_14982_b300 import workloads as W


def _cyclic_case(O, n=(13, 13, 9), A=600.0, eps=0.08):
    """Small curved-wavefront case with four nontrivial SCCs (Eq. curved-state)."""
    g = W.graph_grid(n, A)
    st = W.curved_state(g, W.quarter_source(g), eps)
    _, G, _ = O.metric(g)
    t = O.build_tangent(g, G, st.T, st.s, st.src)
    return g, st, t


def test_dense_bruteforce_primal_and_transpose(oracle_mod):
    """Block traversal (Prop. 3) equals numpy's dense LAPACK solve of A and A^T."""
    O = oracle_mod
    g, st, t = _cyclic_case(O)
    assert np.sum(t.scc_sizes() > 1) == 4
    Ad = t.A().toarray()
    rng = np.random.default_rng(1)
    q = rng.standard_normal((t.N, 3))
    x = O.solve(t, q)
    xd = np.linalg.solve(Ad, q)
    assert np.max(np.abs(x - xd)) <= 1e-12 * np.max(np.abs(xd))
    lam = O.solve_T(t, q)
    ld = np.linalg.solve(Ad.T, q)
    assert np.max(np.abs(lam - ld)) <= 1e-12 * np.max(np.abs(ld))


def test_sparse_lu_agrees_on_table3_grid(oracle_mod):
    """On the 41x41x25 case-C graph (6 SCCs) the traversal agrees with SciPy's sparse LU."""
    O = oracle_mod
    g = W.graph_grid((41, 41, 25), 500.0)
    st = W.curved_state(g, W.quarter_source(g), 0.05)
    _, G, _ = O.metric(g)
    t = O.build_tangent(g, G, st.T, st.s, st.src)
    q = np.random.default_rng(2).standard_normal(t.N)
    x = O.solve(t, q)
    xr = O.direct_solve(t, q)
    assert np.linalg.norm(x - xr) <= 1e-12 * np.linalg.norm(xr)
    lam = O.solve_T(t, q)
    lr = O.direct_solve(t, q, transpose=True)
    assert np.linalg.norm(lam - lr) <= 1e-12 * np.linalg.norm(lr)


def test_scc_partition_matches_scipy(oracle_mod):
    """Tarjan labels give the same partition as scipy.sparse.csgraph strong components."""
    O = oracle_mod
    g = W.graph_grid((41, 41, 25), 500.0)
    st = W.curved_state(g, W.quarter_source(g), 0.05)
    _, G, _ = O.metric(g)
    t = O.build_tangent(g, G, st.T, st.s, st.src)
    j, i = t.edges()
    adj = sp.csr_matrix((np.ones(len(j)), (j, i)), shape=(t.N, t.N))
    nc, lab = connected_components(adj, directed=True, connection="strong")
    assert nc == t.ncomp
    # same partition: the map scipy-label -> oracle-label is a bijection
    pairs = set(zip(lab.tolist(), t.label.tolist()))
    assert len(pairs) == nc
    # oracle label is the smallest node of its component
    for comp in np.unique(t.label):
        assert comp == np.min(np.nonzero(t.label == comp)[0])


def test_prop1_block_triangular_and_levels(oracle_mod):
    """Prop. 1 / Eq. (block-form): in the canonical order every edge goes forward or stays
    inside a component; levels are longest paths (tight)."""
    O = oracle_mod
    g, st, t = _cyclic_case(O)
    pos = np.empty(t.N, dtype=np.int64)
    pos[t.perm] = np.arange(t.N)
    j, i = t.edges()
    cross = t.label[j] != t.label[i]
    assert np.all(pos[j][cross] < pos[i][cross])
    assert np.all(t.level[j][cross] < t.level[i][cross])
    # tightness: a component at level L > 0 has a predecessor at level L - 1
    best = np.full(t.N, -1)
    np.maximum.at(best, t.label[i][cross], t.level[j][cross])
    reps = np.unique(t.label)
    for c in reps:
        if t.level[c] > 0:
            assert best[c] == t.level[c] - 1
        else:
            assert best[c] == -1
    # level_ptr / comp_ptr consistent with perm
    for L in range(t.nlev):
        seg = t.perm[t.level_ptr[L]:t.level_ptr[L + 1]]
        assert np.all(t.level[seg] == L)
    # components ordered by (level, smallest node); nodes ascending inside
    keys = [(t.level[t.perm[a]], t.label[t.perm[a]]) for a in t.comp_ptr[:-1]]
    assert keys == sorted(keys)
    for c in range(t.ncomp):
        seg = t.perm[t.comp_ptr[c]:t.comp_ptr[c + 1]]
        assert np.all(np.diff(seg) > 0) and len(set(t.label[seg])) == 1


def test_prop2_kahn_residual_is_downstream_closure(oracle_mod):
    """Prop. 2: the Kahn residual equals the set reachable from the nontrivial SCCs."""
    O = oracle_mod
    g = W.graph_grid((21, 21, 13), 500.0)
    st = W.curved_state(g, W.quarter_source(g), 0.05)
    _, G, _ = O.metric(g)
    t = O.build_tangent(g, G, st.T, st.s, st.src)
    j, i = t.edges()
    adj = sp.csr_matrix((np.ones(len(j)), (j, i)), shape=(t.N, t.N))
    sizes = dict(zip(*np.unique(t.label, return_counts=True)))
    cyc = np.array([v for v in range(t.N) if sizes[t.label[v]] > 1])
    reach = np.zeros(t.N, dtype=bool)
    for v in cyc:
        if not reach[v]:
            reach[breadth_first_order(adj, v, directed=True, return_predecessors=False)] = True
    assert np.array_equal(~t.kahn_removed(), reach)
    assert reach.sum() == 897


def test_rows_normalized_and_m_matrix(oracle_mod):
    """Eq. (discrete-row): w >= 0, interior rows sum to 1; Theorem (local invertibility):
    A_C^-1 >= 0 for every nontrivial block, so q >= 0 gives dT >= 0."""
    O = oracle_mod
    g, st, t = _cyclic_case(O)
    assert np.all(t.w > 0)
    rs = np.add.reduceat(t.w, t.row_ptr[:-1][np.diff(t.row_ptr) > 0])
    assert np.allclose(rs, 1.0, atol=1e-14)
    for c in range(t.ncomp):
        nodes = t.perm[t.comp_ptr[c]:t.comp_ptr[c + 1]]
        if len(nodes) > 1:
            Ac = O.block_matrix(t, nodes)
            inv = np.linalg.inv(Ac)
            assert np.all(inv >= -1e-14)
            assert np.max(np.abs(np.linalg.eigvals(np.eye(len(nodes)) - Ac))) < 1.0
    q = np.abs(np.random.default_rng(3).standard_normal(t.N))
    assert np.all(O.solve(t, q) >= 0.0)


def test_reversal_criterion_on_violating_edges(oracle_mod):
    """Sec. 5.2.1 / Eq. (reversal): every traveltime-order-violating face has
    T_xi a^xi < 0 (compact normal difference times the face coefficient)."""
    O = oracle_mod
    g = W.graph_grid((41, 41, 25), 600.0)
    st = W.radial_state(g, W.quarter_source(g))
    _, G, _ = O.metric(g)
    t = O.build_tangent(g, G, st.T, st.s, st.src)
    gT = O.grad(g, st.T)
    n = np.array(g.n)
    strides = np.array([n[1] * n[2], n[2], 1])
    j, i = t.edges()
    vio = st.T[j] > st.T[i]
    assert vio.sum() > 0
    for jj, ii in zip(j[vio][:500], i[vio][:500]):
        diff = jj - ii
        d = int(np.nonzero(np.abs(diff) == strides)[0][0])
        sg = 1 if diff > 0 else -1
        gf = 0.5 * (gT[ii] + gT[jj])
        gf[d] = (st.T[jj] - st.T[ii]) / g.dxi[d] * sg
        Gf = 0.5 * (G[ii] + G[jj])
        a = Gf[d] @ gf
        assert gf[d] * a < 0.0
        assert gf[d] * (Gf[d] @ gf - Gf[d, d] * gf[d]) < -Gf[d, d] * gf[d] ** 2 + 1e-30


def test_adjoint_pairing_multisource_2d(oracle_mod):
    """Sec. 4.4 pairing <J p, y> = <p, J^T y> with M, C, P and the source sum (2-D workload,
    constant-gradient closed-form state)."""
    O = oracle_mod
    wl = W.config1()
    g = wl.grid
    _, G, _ = O.metric(g)
    tans = []
    for a, src in enumerate([int(wl.src[0]), g.index(40, 0)]):
        T = W.linear_velocity_T(g.xyz, g.xyz[src], 1.5, 0.5)
        s = 1.0 / (1.5 + 0.5 * g.xyz[:, 1])
        tans.append(O.build_tangent(g, G, T, s, src))
    rng = np.random.default_rng(4)
    p = rng.standard_normal((g.N, 2))
    y = rng.standard_normal((2, len(wl.rec), 2))
    for model in (O.MODEL_SLOWNESS, O.MODEL_VELOCITY, O.MODEL_RELATIVE):
        Jp = O.J(tans, s, wl.rec, p, model=model)
        JTy = O.JT(tans, s, wl.rec, y, model=model)
        l1, l2 = np.sum(Jp * y), np.sum(p * JTy)
        assert abs(l1 - l2) <= 1e-13 * max(abs(l1), abs(l2))


def test_scaling_identity_and_constant_gradient_state(oracle_mod):
    """Sec. 3.2: with q = C(-s), dT = -T exactly; and the tangent of a constant-gradient
    medium is close to the derivative of its closed form under uniform scaling."""
    O = oracle_mod
    wl = W.config1()
    g = wl.grid
    _, G, _ = O.metric(g)
    src = int(wl.src[0])
    T = W.linear_velocity_T(g.xyz, g.xyz[src], 1.5, 0.5)
    s = 1.0 / (1.5 + 0.5 * g.xyz[:, 1])
    t = O.build_tangent(g, G, T, s, src)
    x = O.solve(t, t.cs * (-s))
    assert np.linalg.norm(x + T) <= 1e-14 * np.linalg.norm(T)


def test_directional_sweeping_converges_to_direct(oracle_mod):
    """Sec. 3.6: Gauss-Seidel directional sweeping reaches the block-traversal solution,
    in one cycle when the graph is traveltime ordered on a flat grid."""
    O = oracle_mod
    g, st, t = _cyclic_case(O)
    q = np.random.default_rng(5).standard_normal(t.N)
    x = O.solve(t, q)
    xs, cyc = O.sweep(g, t, q, tol=1e-13)
    assert cyc > 1
    assert np.max(np.abs(xs - x)) <= 1e-11 * np.max(np.abs(x))
    ls, cyc = O.sweep(g, t, q, transpose=True, tol=1e-13)
    lam = O.solve_T(t, q)
    assert np.max(np.abs(ls - lam)) <= 1e-11 * np.max(np.abs(lam))


def test_singular_block_detected(oracle_mod):
    """A 2-cycle with internal row sums exactly 1 violates the theorem's strict-row
    condition; the LU reports a zero pivot."""
    O = oracle_mod
    A = np.array([[1.0, -1.0], [-1.0, 1.0]])
    piv = np.zeros(2, dtype=np.int32)
    assert O.lib().or_lu(2, A.reshape(-1).copy(), piv) == 2


def test_state_homogeneous_fixed_point(oracle_mod):
    """State reading (Sec. 2.1-2.2): in a homogeneous medium tau = 1 is the discrete fixed
    point, so T = s |x - x_s| on the deformed grid to rounding, after one cycle."""
    O = oracle_mod
    g = W.table1_grid(21)
    src = g.index(10, 10, 0)
    T, cyc = O.eik_forward(g, np.full(g.N, 1.0 / 3000.0), src)
    ref = np.sqrt(((g.xyz - g.xyz[src]) ** 2).sum(1)) / 3000.0
    assert cyc == 1 and np.max(np.abs(T - ref)) <= 1e-15


def test_state_first_order_on_skewed_box(oracle_mod):
    """State reading: against the constant-gradient closed form on a convex box with a
    non-orthogonal interior map the max error halves with h (first order)."""
    O = oracle_mod
    errs = []
    for m in (1, 2, 4):
        g = W.skew_box_grid((30 * m + 1, 20 * m + 1))
        v = 1.5 + 0.5 * g.xyz[:, 1]
        src = g.index(10 * m, 5 * m)
        T, cyc = O.eik_forward(g, 1.0 / v, src)
        assert cyc > 0
        Tex = W.linear_velocity_T(g.xyz, g.xyz[src], 1.5, 0.5)
        errs.append(np.max(np.abs(T - Tex)) / Tex.max())
    assert errs[0] < 0.03
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.3


def test_state_converges_on_topography_3d(oracle_mod):
    """State reading: the sweeping converges on a 3-D workload recipe with topography."""
    O = oracle_mod
    g, _ = W._config3d("3d", (41, 41, 21), 20.0, 8.0, 2.0, 20263)
    s = 1.0 / W._velocity3d(g, 2.0)
    T, cyc = O.eik_forward(g, s, g.index(10, 10, 0))
    assert 0 < cyc < 100 and np.all(T >= 0) and np.isfinite(T).all()


def test_closed_cycle_block_is_singular(oracle_mod):
    """A state with a closed cyclic component (no upwind face leaves it): its rows of W
    sum to 1, so A_C = I - W_CC has the all-ones null vector; the oracle's LU reports the
    zero pivot and its tangent build refuses the state (Sec. 4.2, local invertibility)."""
    import pytest
    O = oracle_mod
    g, T, s, src = W.closed_cycle_case()
    _, G, _ = O.metric(g)
    t = O.assemble(g, G, T, s, src)
    lab = np.zeros(g.N, dtype=np.int32)
    O.lib().or_scc(g.N, t.row_ptr, t.col, lab)
    vals, counts = np.unique(lab, return_counts=True)
    closed = []
    for v, c in zip(vals, counts):
        nodes = np.nonzero(lab == v)[0]
        inside = set(nodes.tolist())
        if c > 1 and all(int(t.col[e]) in inside for i in nodes for e in range(t.row_ptr[i], t.row_ptr[i + 1])):
            closed.append(nodes)
    assert len(closed) == 1 and len(closed[0]) == 4
    Ac = O.block_matrix(t, closed[0])
    assert np.max(np.abs(Ac @ np.ones(4))) <= 1e-15          # rows of W_CC sum to 1
    piv = np.zeros(4, dtype=np.int32)
    assert O.lib().or_lu(4, np.ascontiguousarray(Ac.reshape(-1)).copy(), piv) != 0
    with pytest.raises(np.linalg.LinAlgError):
        O.build_tangent(g, G, T, s, src)
