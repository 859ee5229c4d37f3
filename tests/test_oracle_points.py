"""Oracle pins for off-grid point sources: the state from the interpolated source
slowness, the differentiated seed rows of Sec. 3.1-3.2 and the direct term D_a of
Sec. 4.4 (Eq. source-jacobian), checked against closed forms, the exact scaling
identity, a finite-difference derivative of the oracle's own state solve, and the
adjoint pairing."""
import numpy as np
import scipy.sparse as sp

from paper_2609_14982_b300 import workloads as W


def _bilinear_grid(n, c=(0.15, -0.1)):
    """Mapped grid whose top surface is a plane, zsurf = c . (x, y): the map
    z = zeta + (1 - zeta/H) zsurf is multilinear in the logical coordinates, so a
    point's physical position is the map itself at its fractional coordinates."""
    if len(n) == 2:
        return W.mapped_grid(n, (0.0,), (2.0 * (n[0] - 1),), 1.0 * (n[1] - 1), lambda x: c[0] * x)
    return W.mapped_grid(n, (0.0, 0.0), (2.0 * (n[0] - 1), 1.5 * (n[1] - 1)), 1.0 * (n[2] - 1),
                         lambda x, y: c[0] * x + c[1] * y)


def _map_point(g, f, c=(0.15, -0.1)):
    nd = g.ndim
    h = [2.0, 1.5][:nd - 1]
    xs = [g.lo[d] + f[d] * h[d] for d in range(nd - 1)]
    zeta = f[-1] * 1.0
    H = 1.0 * (g.n[-1] - 1)
    zs = sum(c[d] * xs[d] for d in range(nd - 1))
    return np.array(xs + [zeta + (1.0 - zeta / H) * zs])


def test_point_source_homogeneous_state_is_exact(oracle_mod):
    """In a homogeneous medium tau = 1 is the fixed point, so T = s |x - x_src| at every
    node, with x_src the grid map at the source's fractional coordinates (2-D and 3-D)."""
    O = oracle_mod
    for n, f in (((21, 13), (7.3, 4.6)), ((11, 9, 7), (3.25, 5.5, 2.75))):
        g = _bilinear_grid(n)
        s = np.full(g.N, 0.5)
        T, cyc, ps = O.eik_forward_point(g, s, f)
        xs = _map_point(g, f)
        assert np.max(np.abs(ps.x - xs)) <= 1e-12 * np.max(np.abs(xs))
        ref = 0.5 * np.sqrt(((g.xyz - xs) ** 2).sum(1))
        assert cyc >= 1 and np.max(np.abs(T - ref)) <= 1e-12 * ref.max()
        assert abs(ps.s_src - 0.5) <= 1e-15 and abs(ps.phi.sum() - 1.0) <= 1e-15


def test_point_source_state_first_order_on_skewed_box(oracle_mod):
    """Constant-gradient medium on the non-orthogonal box: the point-source state
    converges to the closed form at first order (the error halves with h)."""
    O = oracle_mod
    errs = []
    for m in (1, 2, 4):
        g = W.skew_box_grid((30 * m + 1, 20 * m + 1))
        v = 1.5 + 0.5 * g.xyz[:, 1]
        T, cyc, ps = O.eik_forward_point(g, 1.0 / v, (10.4 * m, 5.7 * m))
        assert cyc > 0
        Tex = W.linear_velocity_T(g.xyz, ps.x, 1.5, 0.5)
        errs.append(np.max(np.abs(T - Tex)) / Tex.max())
    assert errs[0] < 0.03
    for a, b in zip(errs, errs[1:]):
        assert 1.7 < a / b < 2.4


def _case(O, n=(31, 21), f=(9.4, 6.35), model=None):
    g = W.skew_box_grid(n)
    v = 1.5 + 0.5 * g.xyz[:, 1] + 0.1 * np.sin(g.xyz[:, 0])
    s = 1.0 / v
    T, cyc, ps = O.eik_forward_point(g, s, f)
    assert cyc > 0
    _, G, _ = O.metric(g)
    t = O.build_tangent_point(g, G, T, s, ps)
    return g, s, T, ps, t


def test_point_source_seed_rows(oracle_mod):
    """The seed rows are the cell corners, identities with c = 0, and every corner keeps
    T = s_src r in the state."""
    O = oracle_mod
    g, s, T, ps, t = _case(O)
    assert len(ps.nodes) == 4 and len(set(ps.nodes.tolist())) == 4
    for k, i in enumerate(ps.nodes):
        assert t.row_type[i] == 1 and t.cs[i] == 0.0 and t.row_ptr[i + 1] == t.row_ptr[i]
        assert abs(T[i] - ps.s_src * ps.r[k]) <= 1e-15 * T[i]
    assert int((t.row_type == 1).sum()) == 4


def test_point_source_scaling_identity(oracle_mod):
    """Sec. 3.2's identity through the differentiated seed rows: dv = v, i.e. ds = -s,
    gives dT = -T at every node (seed corners included), by the block traversal and by
    the assembled direct solve."""
    O = oracle_mod
    g, s, T, ps, t = _case(O)
    q = O.source_rhs(t, (-s)[:, None])
    for x in (O.solve(t, q), O.direct_solve(t, q)):
        assert np.max(np.abs(x[:, 0] + T)) <= 1e-12 * T.max()
    # through J with the relative model (m = 1 means dv = v)
    rec = np.arange(0, g.N, 7)
    d = O.J([t], s, rec, np.ones((g.N, 1)), model=O.MODEL_RELATIVE)
    assert np.max(np.abs(d[0, :, 0] + T[rec])) <= 1e-12 * T.max()


def test_point_source_seed_rows_are_the_state_derivative(oracle_mod):
    """Each seed corner's T = s_src(s) r is linear in the corner slownesses, so central
    differences of the oracle's own state solve give dT_o/ds_k = r_o phi_k exactly (up
    to rounding); J's seed rows (slowness model, p = e_k) must equal them for every k."""
    O = oracle_mod
    g, s, T, ps, t = _case(O, n=(21, 15), f=(6.3, 4.8))
    h = 1e-4
    for k in ps.nodes:
        e = np.zeros(g.N)
        e[k] = 1.0
        Tp, _, _ = O.eik_forward_point(g, s + h * e, ps.f)
        Tm, _, _ = O.eik_forward_point(g, s - h * e, ps.f)
        fd = (Tp[ps.nodes] - Tm[ps.nodes]) / (2 * h)
        jd = O.J([t], s, ps.nodes, e[:, None])[0, :, 0]
        assert np.max(np.abs(fd - jd)) <= 1e-9 * np.max(np.abs(jd)), k


def test_point_source_adjoint_pairing(oracle_mod):
    """<J p, y> = <p, J^T y> with point and node sources mixed, velocity model."""
    O = oracle_mod
    g, s, T, ps, t = _case(O)
    _, G, _ = O.metric(g)
    src2 = g.index(20, 3)
    T2, _ = O.eik_forward(g, s, src2)
    t2 = O.build_tangent(g, G, T2, s, src2)
    rng = np.random.default_rng(3)
    rec = rng.choice(g.N, 40, replace=False)
    p = rng.standard_normal((g.N, 3))
    y = rng.standard_normal((2, len(rec), 3))
    d = O.J([t, t2], s, rec, p, model=O.MODEL_VELOCITY)
    gT = O.JT([t, t2], s, rec, y, model=O.MODEL_VELOCITY)
    l1, l2 = float((d * y).sum()), float((p * gT).sum())
    assert abs(l1 - l2) <= 1e-12 * max(abs(l1), abs(l2))


def test_direct_term_for_receivers_in_the_source_cell(oracle_mod):
    """D_a (reading): a receiver inside the source cell is predicted as s_src |x_r - x_src|,
    so its Jacobian row is |x_r - x_src| phi (closed form: s_src is linear in the corner
    slownesses); receivers elsewhere have a zero D row; with P's direct rows zeroed the
    interpolated J and J^T keep the adjoint pairing."""
    O = oracle_mod
    g, s, T, ps, t = _case(O)
    f_rec = np.array([[9.8, 6.1], [9.0, 6.9], [9.4, 6.35], [15.5, 12.25], [3.2, 17.0]])
    D, direct = O.direct_term(g, ps, f_rec)
    assert direct.tolist() == [True, True, True, False, False]
    # row of a direct receiver against the closed form: d(s_src rho)/ds_k = rho phi_k
    P = O.receiver_interp(g, f_rec)
    Pm = sp.diags((~direct).astype(float)) @ P
    for j in range(3):
        xr = np.asarray(P[j] @ g.xyz).ravel()
        rho = np.sqrt(((xr - ps.x) ** 2).sum())
        row = np.asarray(D[j].todense()).ravel()
        assert np.allclose(row[ps.nodes], rho * ps.phi, rtol=0, atol=1e-15 * max(rho, 1.0))
        assert np.count_nonzero(row) <= len(ps.nodes)
    assert D[3:].nnz == 0
    assert abs(float((D[2] @ np.ones(g.N))[0])) <= 1e-12   # the receiver at the source point
    rng = np.random.default_rng(5)
    p = rng.standard_normal((g.N, 2))
    y = rng.standard_normal((1, len(f_rec), 2))
    d = O.J_interp([t], s, [Pm], p, Ds=[D])
    gT = O.JT_interp([t], s, [Pm], y, Ds=[D])
    l1, l2 = float((d * y).sum()), float((p * gT).sum())
    assert abs(l1 - l2) <= 1e-12 * max(abs(l1), abs(l2))
    # the direct receivers depend on the model only through the source cell's corners
    q = np.zeros((g.N, 1))
    q[ps.nodes[0], 0] = 1.0
    dj = O.J_interp([t], s, [Pm], q, Ds=[D])[0, :3, 0]
    for j in range(3):
        xr = np.asarray(P[j] @ g.xyz).ravel()
        assert abs(dj[j] - np.sqrt(((xr - ps.x) ** 2).sum()) * ps.phi[0]) <= 1e-15
