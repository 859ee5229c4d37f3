"""Oracle of the augmented Gauss-Newton system (Sec. 4.5) pinned to other mathematics:
LSMR against SciPy's independent implementation and against the exact least-squares
solution, its norm recurrences against the true norms, the roughness operator against
networkx's grid-graph Laplacian, and the augmented solve against the normal equations
of Eq. (gn-subproblem)."""
import networkx as nx
import numpy as np
import scipy.sparse.linalg as sla

from paper_2609_14982_b300 import workloads as W


def test_lsmr_matches_scipy_iterates_and_norms(oracle_mod):
    """Same iterate as scipy.sparse.linalg.lsmr after k steps; the carried |r_k| equals
    |b - A x_k| and |zetabar| equals |A^T r_k| (the quantity LSMR minimizes)."""
    rng = np.random.default_rng(0)
    A = rng.standard_normal((40, 15))
    b = rng.standard_normal(40)
    for k in (1, 2, 3, 7, 15):
        x, info = oracle_mod.lsmr(lambda v: A @ v, lambda u: A.T @ u, b, k)
        xs = sla.lsmr(A, b, atol=0.0, btol=0.0, conlim=0.0, maxiter=k)[0]
        assert np.max(np.abs(x - xs)) <= 1e-12 * np.max(np.abs(xs))
        r = b - A @ x
        assert abs(info["normr"] - np.linalg.norm(r)) <= 1e-12 * np.linalg.norm(b)
        assert abs(info["normar"] - np.linalg.norm(A.T @ r)) <= 1e-11 * np.linalg.norm(A.T @ b)
        assert abs(info["normx"] - np.linalg.norm(x)) <= 1e-14 * np.linalg.norm(x)
    # after n steps (exact arithmetic: the minimizer) the least-squares solution
    xe = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.max(np.abs(x - xe)) <= 1e-10 * np.max(np.abs(xe))


def test_lsmr_norm_ar_decreases_monotonically(oracle_mod):
    """|A^T r_k| is nonincreasing in k (the defining property of LSMR), also for a
    rank-deficient, ill-conditioned matrix."""
    rng = np.random.default_rng(3)
    U = rng.standard_normal((60, 20))
    A = U @ np.diag(np.logspace(0, -6, 20)) @ rng.standard_normal((20, 25))
    b = rng.standard_normal(60)
    prev = np.inf
    for k in range(1, 30):
        _, info = oracle_mod.lsmr(lambda v: A @ v, lambda u: A.T @ u, b, k)
        assert info["normar"] <= prev * (1 + 1e-9)
        prev = info["normar"]


def test_roughness_is_first_differences_and_grid_laplacian(oracle_mod):
    """R p of a linear function is its slope per axis; R^T R is the graph Laplacian of the
    logical grid (networkx), so R is one difference per adjacent node pair."""
    n = (5, 4, 3)
    g = W.Grid(3, n, (1.0, 1.0, 1.0), np.zeros((int(np.prod(n)), 3)))
    Rm = oracle_mod.roughness(g)
    assert Rm.shape == (4 * 4 * 3 + 5 * 3 * 3 + 5 * 4 * 2, 60)
    i, j, k = np.meshgrid(*[np.arange(m) for m in n], indexing="ij")
    p = (3.0 * i + 5.0 * j + 7.0 * k).ravel()
    Rp = Rm @ p
    assert np.all(Rp[:48] == 3.0) and np.all(Rp[48:93] == 5.0) and np.all(Rp[93:] == 7.0)
    G = nx.grid_graph(dim=[range(m) for m in n])
    sizes = [max(t[d] for t in G.nodes) + 1 for d in range(3)]
    perm = [sizes.index(m) for m in n]          # tuple position of each of our axes
    order = sorted(G.nodes, key=lambda t: (t[perm[0]] * n[1] + t[perm[1]]) * n[2] + t[perm[2]])
    L = nx.laplacian_matrix(G, nodelist=order).toarray()
    assert np.array_equal((Rm.T @ Rm).toarray(), L)


def _gn_case(O):
    """Two sources on a small curved-surface 3-D grid, velocity model, receivers on every
    second surface node."""
    g = W.graph_grid((9, 9, 5), 300.0)
    _, G, _ = O.metric(g)
    tans = []
    for src in (W.quarter_source(g), W.centre_source(g)):
        st = W.curved_state(g, src, 0.05)
        tans.append(O.build_tangent(g, G, st.T, st.s, st.src))
    s = st.s
    rec = np.array([g.index(i, j, 0) for i in range(0, 9, 2) for j in range(0, 9, 2)], dtype=np.int64)
    return g, tans, s, rec


def test_gn_operator_adjoint_and_normal_equations(oracle_mod):
    """<K p, y> = <p, K^T y>, and LSMR on the augmented system reaches the minimizer of
    Eq. (gn-subproblem), i.e. the solution of
    (J^T W_d^2 J + lam^2 R^T R + lam^2 S^2) dv = -J^T W_d^2 r  (dense numpy solve)."""
    O = oracle_mod
    g, tans, s, rec = _gn_case(O)
    rng = np.random.default_rng(5)
    N, S_ = g.N, len(tans)
    vk = 1.0 / s
    wd = 1.0 / (0.0003 + 0.003 * rng.uniform(0.5, 1.5, (S_, len(rec))))
    lam, gamma = 0.5, 1.0
    K, KT, m = O.gn_operator(g, tans, s, rec, wd, vk, lam, gamma)
    p, y = rng.standard_normal(N), rng.standard_normal(m)
    l1, l2 = float(K(p) @ y), float(p @ KT(y))
    assert abs(l1 - l2) <= 1e-12 * max(abs(l1), abs(l2))
    # dense J (columns = J e_j) and the normal equations
    Jd = O.J(tans, s, rec, np.eye(N), model=O.MODEL_VELOCITY).reshape(S_ * len(rec), N)
    Rm = O.roughness(g).toarray()
    Wd = wd.ravel()
    r = rng.standard_normal(S_ * len(rec)) * 1e-3
    H = Jd.T @ (Wd[:, None] ** 2 * Jd) + lam ** 2 * (Rm.T @ Rm) + lam ** 2 * np.diag((gamma / vk) ** 2)
    dv_ne = np.linalg.solve(H, -Jd.T @ (Wd ** 2 * r))
    b = np.concatenate([-Wd * r, np.zeros(m - len(Wd))])
    dv, info = O.lsmr(K, KT, b, 400)
    assert np.max(np.abs(dv - dv_ne)) <= 1e-7 * np.max(np.abs(dv_ne))
    assert info["normar"] <= 1e-9 * info["norma"] * info["normr"]


def test_gn_operator_on_cells_normal_equations(oracle_mod):
    """The same minimizer check with the model on cells: LSMR on K_cells reaches the
    solution of (A^T J^T W_d^2 J A + lam^2 R_c^T R_c + lam^2 S_c^2) dv = -A^T J^T W_d^2 r."""
    O = oracle_mod
    g, tans, s, rec = _gn_case(O)
    rng = np.random.default_rng(8)
    A = O.cell_average(g)
    nc = A.shape[1]
    vc = 2.0 + rng.uniform(0.0, 0.5, nc)
    wd = 1.0 / (0.0003 + 0.003 * rng.uniform(0.5, 1.5, (len(tans), len(rec))))
    lam, gamma = 0.5, 1.0
    K, KT, m = O.gn_operator(g, tans, s, rec, wd, vc, lam, gamma, cells=True)
    p, y = rng.standard_normal(nc), rng.standard_normal(m)
    l1, l2 = float(K(p) @ y), float(p @ KT(y))
    assert abs(l1 - l2) <= 1e-12 * max(abs(l1), abs(l2))
    Jd = O.J(tans, s, rec, np.asarray(A.todense()), model=O.MODEL_VELOCITY).reshape(len(tans) * len(rec), nc)
    cg = W.Grid(3, tuple(x - 1 for x in g.n), g.dxi, np.zeros((nc, 3)))
    Rc = O.roughness(cg).toarray()
    Wd = wd.ravel()
    r = rng.standard_normal(Wd.size) * 1e-3
    H = Jd.T @ (Wd[:, None] ** 2 * Jd) + lam ** 2 * (Rc.T @ Rc) + lam ** 2 * np.diag((gamma / vc) ** 2)
    dv_ne = np.linalg.solve(H, -Jd.T @ (Wd ** 2 * r))
    b = np.concatenate([-Wd * r, np.zeros(m - Wd.size)])
    dv, info = O.lsmr(K, KT, b, 400)
    assert np.max(np.abs(dv - dv_ne)) <= 1e-7 * np.max(np.abs(dv_ne))
