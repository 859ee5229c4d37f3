"""GPU: off-grid point sources through the C ABI against the oracle -- the state of
eik_forward_points, the tangent of tangent_build_points (structure bit for bit, seed
rows), J p and J^T y with the differentiated seed rows (on-grid receivers, the full dT
field, per-source and summed transposes, column chunks, both schedules), the scaling
identity, and off-grid receivers inside the source cell carried by the direct term D_a
(Sec. 3.1-3.2, Sec. 4.4 Eq. source-jacobian / source-transpose)."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _grid2d():
    g = W.skew_box_grid((41, 29))
    v = 1.5 + 0.5 * g.xyz[:, 1] + 0.1 * np.sin(g.xyz[:, 0])
    return g, 1.0 / v, np.array([[12.4, 8.65], [30.0, 3.5], [21.7, 20.2]])


def _grid3d():
    g = W.graph_grid((21, 21, 13), 500.0)
    s = W.curved_state(g, g.index(5, 5, 0), 0.05).s
    return g, s, np.array([[5.3, 4.6, 0.4], [14.5, 10.25, 2.75]])


@pytest.fixture(scope="module", params=["2d", "3d"])
def case(request, oracle_mod):
    g, s, f = _grid2d() if request.param == "2d" else _grid3d()
    O = oracle_mod
    res = [O.eik_forward_point(g, s, fa) for fa in f]
    Ts = np.stack([r[0] for r in res])
    pss = [r[2] for r in res]
    _, G, _ = O.metric(g)
    otans = [O.build_tangent_point(g, G, Ts[a], s, pss[a]) for a in range(len(f))]
    rng = np.random.default_rng(8)
    corners = [int(pss[a].nodes[1]) for a in range(len(f))]          # a receiver on a seed corner
    rec = np.unique(np.concatenate([corners, rng.choice(g.N, 40, replace=False)])).astype(np.int32)
    return g, s, f, Ts, pss, otans, rec


def _tangent(g, s, f, Ts, rec, **opts):
    return eik.Tangent(eik.DeviceGrid(g), torch.tensor(Ts, device=DEV), torch.tensor(s, device=DEV), f, rec=rec,
                       opts=eik.default_opts(**opts), points=True)


def _rel(a, b):
    a = a.double().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_point_state_matches_oracle(case):
    g, s, f, Ts, pss, otans, rec = case
    T, cyc = eik.eik_forward_points(eik.DeviceGrid(g), torch.tensor(s, device=DEV), f)
    assert cyc > 0
    assert _rel(T, Ts) <= 1e-12
    for a, ps in enumerate(pss):      # every seed corner holds s_src r exactly
        assert np.max(np.abs(T[a].cpu().numpy()[ps.nodes] - ps.s_src * ps.r)) <= 1e-14 * Ts[a].max()


def test_point_state_homogeneous_exact():
    g = W.mapped_grid((21, 13), (0.0,), (40.0,), 12.0, lambda x: 0.15 * x)
    T, _ = eik.eik_forward_points(eik.DeviceGrid(g), torch.full((g.N,), 0.5, device=DEV, dtype=torch.float64),
                                  [[7.3, 4.6]])
    xs = np.array([7.3 * 2.0, 4.6 + (1 - 4.6 / 12.0) * 0.15 * 7.3 * 2.0])
    ref = 0.5 * np.sqrt(((g.xyz - xs) ** 2).sum(1))
    assert _rel(T[0], ref) <= 1e-12


def test_point_tangent_structure_matches_oracle(case):
    g, s, f, Ts, pss, otans, rec = case
    tan = _tangent(g, s, f, Ts, rec)
    for a, ot in enumerate(otans):
        ex = tan.export(a)
        assert np.array_equal(ex["label"], ot.label) and np.array_equal(ex["perm"], ot.perm)
        assert np.array_equal(ex["level_ptr"], ot.level_ptr)
        assert np.all(ex["cs"][pss[a].nodes] == 0.0)
        assert np.max(np.abs(ex["cs"] - ot.cs)) <= 1e-12 * np.max(np.abs(ot.cs))


@pytest.mark.parametrize("model", ["slowness", "velocity"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_point_jacobian_against_oracle(oracle_mod, case, model, dtype):
    """J p (shared model: receivers and the full dT field) and J^T y (summed and per source)
    with the seed rows, against the oracle."""
    O = oracle_mod
    g, s, f, Ts, pss, otans, rec = case
    mcode = eik.MODEL_SLOWNESS if model == "slowness" else eik.MODEL_VELOCITY
    ocode = O.MODEL_SLOWNESS if model == "slowness" else O.MODEL_VELOCITY
    tan = _tangent(g, s, f, Ts, rec, model=mcode)
    rng = np.random.default_rng(17)
    R = 8
    p = torch.tensor(rng.standard_normal((g.N, R)), device=DEV, dtype=dtype)
    y = torch.tensor(rng.standard_normal((len(f), len(rec), R)), device=DEV, dtype=dtype)
    dT = torch.empty((len(f), g.N, R), device=DEV, dtype=dtype)
    _, drec = tan.apply(p, shared_model=True, dT_full=dT)
    gs, _ = tan.apply_T(y, sum_sources=True)
    ga, _ = tan.apply_T(y, sum_sources=False)
    tan.status()
    tol = 1e-10 if dtype == torch.float64 else 1e-5
    pn, yn = p.double().cpu().numpy(), y.double().cpu().numpy()
    assert _rel(drec, O.J(otans, s, rec, pn, model=ocode)) <= tol
    full = O.J(otans, s, np.arange(g.N), pn, model=ocode)
    assert _rel(dT, full) <= tol
    assert _rel(gs, O.JT(otans, s, rec, yn, model=ocode)) <= tol
    assert _rel(ga, O.JT(otans, s, rec, yn, model=ocode, sum_sources=False)) <= tol


def test_point_scaling_identity(case):
    """ds = -s (slowness model) gives dT = -T at every node, seed corners included."""
    g, s, f, Ts, pss, otans, rec = case
    tan = _tangent(g, s, f, Ts, rec)
    p = torch.tensor(-s, device=DEV).unsqueeze(1).contiguous()
    dT = torch.empty((len(f), g.N, 1), device=DEV, dtype=torch.float64)
    tan.apply(p, shared_model=True, dT_full=dT)
    tan.status()
    assert float((dT[..., 0].cpu() + torch.tensor(Ts)).abs().max()) <= 1e-12 * Ts.max()


def test_point_schedules_and_chunks_agree(case):
    """The seed terms are outside the traversal: persistent and cluster schedules give the
    same bits, and column chunks of 2 the same bits as one pass."""
    g, s, f, Ts, pss, otans, rec = case
    rng = np.random.default_rng(4)
    p = torch.tensor(rng.standard_normal((g.N, 8)), device=DEV)
    y = torch.tensor(rng.standard_normal((len(f), len(rec), 8)), device=DEV)
    outs = []
    for kw in ({}, {"schedule": eik.SCHED_CLUSTER}, {"rhs_chunk": 2}):
        tan = _tangent(g, s, f, Ts, rec, **kw)
        _, drec = tan.apply(p, shared_model=True)
        gs, _ = tan.apply_T(y, sum_sources=True)
        tan.status()
        outs.append((drec, gs))
        tan.free()
    for o in outs[1:]:
        assert torch.equal(o[0], outs[0][0]) and torch.equal(o[1], outs[0][1])


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_point_direct_term_interp_receivers(oracle_mod, case, dtype):
    """Off-grid receivers, three of them in each source's cell (carried by D_a) and the rest
    elsewhere (multilinear P): J p and J^T y against the oracle's (P A^-1 C + D) M."""
    O = oracle_mod
    g, s, f, Ts, pss, otans, rec = case
    rng = np.random.default_rng(23)
    nd = g.ndim
    n_ip = 12
    fr = np.empty((len(f), n_ip, nd))
    for a in range(len(f)):
        base = np.minimum(np.floor(f[a]), np.array(g.n[:nd]) - 2)
        fr[a, :3] = base + rng.uniform(0.05, 0.95, (3, nd))
        fr[a, 3] = f[a]                              # a receiver at the source point itself
        fr[a, 4:] = rng.uniform(0, 1, (n_ip - 4, nd)) * (np.array(g.n[:nd]) - 1)
    tan = _tangent(g, s, f, Ts, rec)
    tan.set_receivers(fr)
    Ps, Ds = [], []
    for a in range(len(f)):
        D, direct = O.direct_term(g, pss[a], fr[a])
        assert direct[:4].all()
        P = O.receiver_interp(g, fr[a])
        Ps.append(sp.diags((~direct).astype(float)) @ P)
        Ds.append(D)
    p = torch.tensor(rng.standard_normal((g.N, 4)), device=DEV, dtype=dtype)
    y = torch.tensor(rng.standard_normal((len(f), n_ip, 4)), device=DEV, dtype=dtype)
    d = tan.apply_interp(p)
    gT = tan.apply_interp_T(y)
    tan.status()
    tol = 1e-10 if dtype == torch.float64 else 1e-5
    pn, yn = p.double().cpu().numpy(), y.double().cpu().numpy()
    assert _rel(d, O.J_interp(otans, s, Ps, pn, Ds=Ds)) <= tol
    assert _rel(gT, O.JT_interp(otans, s, Ps, yn, Ds=Ds)) <= tol


def test_point_tangent_refused_by_batch(case):
    g, s, f, Ts, pss, otans, rec = case
    tan = _tangent(g, s, f, Ts, rec)
    p = torch.zeros((g.N, 4), device=DEV)
    with pytest.raises(eik.EikError):
        eik.apply_batch([tan], [p])


def test_point_source_outside_grid_refused(case):
    g, s, f, Ts, pss, otans, rec = case
    bad = f.copy()
    bad[0, 0] = g.n[0] - 0.5
    with pytest.raises(eik.EikError):
        eik.eik_forward_points(eik.DeviceGrid(g), torch.tensor(s, device=DEV), bad)
