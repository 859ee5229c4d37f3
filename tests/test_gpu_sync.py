"""GPU parity of the level-synchronous schedule (one cooperative launch, every source one
level per global step, a grid-wide barrier between steps, SCC blocks in two steps): the
bare solves A^-1 q, A^-T r and the Jacobian actions against the CPU FP64 oracle, and
bit-for-bit equality with the persistent schedule, which runs the same per-node
arithmetic in the same order."""
import numpy as np
import pytest
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-10, torch.float32: 1e-5}
DEV = "cuda"


def rel_err(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300))


def _graph_case(n, A, eps, srcs):
    g = W.graph_grid(n, A)
    Ts = [W.curved_state(g, g.index(a, b, 0), eps).T for (a, b) in srcs]
    s = W.curved_state(g, g.index(*srcs[0], 0), eps).s
    return g, np.stack(Ts), s, np.array([g.index(a, b, 0) for (a, b) in srcs], dtype=np.int32)


def _config1_case():
    wl = W.config1()
    g = wl.grid
    srcs = [int(wl.src[0]), g.index(45, 0)]
    s = 1.0 / (1.5 + 0.5 * g.xyz[:, 1])
    Ts = np.stack([W.linear_velocity_T(g.xyz, g.xyz[k], 1.5, 0.5) for k in srcs])
    return g, Ts, s, np.array(srcs, dtype=np.int32)


CASES = {
    "cyclic-13x13x9": lambda: _graph_case((13, 13, 9), 600.0, 0.08, [(3, 3), (6, 6), (9, 3)]),
    "table3-41x41x25": lambda: _graph_case((41, 41, 25), 500.0, 0.05, [(10, 10), (20, 20), (30, 10)]),
    "config1-2d": _config1_case,
}


@pytest.fixture(scope="module")
def case(oracle_mod):
    cache = {}

    def get(name):
        if name not in cache:
            g, Ts, s, srcs = CASES[name]()
            _, G, _ = oracle_mod.metric(g)
            otans = [oracle_mod.build_tangent(g, G, Ts[a], s, int(srcs[a])) for a in range(len(srcs))]
            cache[name] = (g, Ts, s, srcs, otans)
        return cache[name]

    return get


def _tangent(g, Ts, s, srcs, rec=None, **kw):
    opts = eik.default_opts(schedule=eik.SCHED_SYNC, **kw)
    return eik.Tangent(eik.DeviceGrid(g), torch.tensor(Ts, device=DEV), torch.tensor(s, device=DEV), srcs,
                       rec=rec, opts=opts)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("R", [1, 3, 8, 64])
def test_sync_solves_against_oracle(oracle_mod, case, name, dtype, R):
    """A^-1 q and A^-T r of every source (Prop. 3, Sec. 4.3) against the oracle's direct
    block solve; the cases hold nontrivial SCC blocks (two steps each in this schedule)."""
    g, Ts, s, srcs, otans = case(name)
    tan = _tangent(g, Ts, s, srcs)
    S, N = len(srcs), g.N
    rng = np.random.default_rng(200 + R)
    qd = torch.tensor(rng.standard_normal((S, N, R)), device=DEV, dtype=dtype)
    x = tan.solve(qd).double().cpu().numpy()
    lam = tan.solve_T(qd).double().cpu().numpy()
    tan.status()
    qq = qd.double().cpu().numpy()
    for a in range(S):
        assert rel_err(x[a], oracle_mod.solve(otans[a], qq[a])) <= TOL[dtype]
        assert rel_err(lam[a], oracle_mod.solve_T(otans[a], qq[a])) <= TOL[dtype]


@pytest.mark.parametrize("units", [0, 2, 4])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_sync_matches_persistent_bitwise(case, units, dtype):
    """Every thread shape (1024 threads x 1 task, 768 x 2, 512 x 4 in flight) gives
    exactly the persistent schedule's result: each node is the same sum in the same
    order, and each SCC block row the same FP64 dot product with A_C^-1."""
    g, Ts, s, srcs, _ = case("table3-41x41x25")
    S, N, R = len(srcs), g.N, 64
    rng = np.random.default_rng(7)
    qd = torch.tensor(rng.standard_normal((S, N, R)), device=DEV, dtype=dtype)
    ref_t = eik.Tangent(eik.DeviceGrid(g), torch.tensor(Ts, device=DEV), torch.tensor(s, device=DEV), srcs)
    ref_x, ref_l = ref_t.solve(qd), ref_t.solve_T(qd)
    tan = _tangent(g, Ts, s, srcs, pass_units=units)
    x, lam = tan.solve(qd), tan.solve_T(qd)
    tan.status()
    assert tan.stats(0)["nontrivial"] + tan.stats(1)["nontrivial"] + tan.stats(2)["nontrivial"] > 0
    assert torch.equal(x, ref_x)
    assert torch.equal(lam, ref_l)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("model", [eik.MODEL_SLOWNESS, eik.MODEL_VELOCITY])
def test_sync_jacobian_actions_against_oracle(oracle_mod, case, dtype, model):
    """J p = P A^-1 C M p (shared model, receivers sampled in the traversal) and
    J^T y = sum_a M^T C^T A_a^-T P^T y_a (Sec. 4.4) against the oracle, with the full
    natural-order fields written on request."""
    g, Ts, s, srcs, otans = case("cyclic-13x13x9")
    S, N, R = len(srcs), g.N, 8
    rec = np.array([g.index(i, j, 0) for i in range(0, 13, 2) for j in range(0, 13, 3)], dtype=np.int32)
    tan = _tangent(g, Ts, s, srcs, rec=rec, model=model)
    rng = np.random.default_rng(3)
    p = torch.tensor(rng.standard_normal((N, R)), device=DEV, dtype=dtype)
    y = torch.tensor(rng.standard_normal((S, len(rec), R)), device=DEV, dtype=dtype)
    dT = torch.empty((S, N, R), device=DEV, dtype=dtype)
    _, jp = tan.apply(p, shared_model=True, dT_full=dT)
    g_sum, _ = tan.apply_T(y, sum_sources=True)
    g_each, _ = tan.apply_T(y, sum_sources=False)
    tan.status()
    pp, yy = p.double().cpu().numpy(), y.double().cpu().numpy()
    ref_jp = oracle_mod.J(otans, s, rec, pp, model=model)
    ref_jt = oracle_mod.JT(otans, s, rec, yy, model=model)
    assert rel_err(jp.double().cpu().numpy(), ref_jp) <= TOL[dtype]
    assert rel_err(g_sum.double().cpu().numpy(), ref_jt) <= TOL[dtype]
    assert rel_err(g_each.double().cpu().numpy().sum(axis=0), ref_jt) <= TOL[dtype]
    for a in range(S):
        assert np.array_equal(dT[a].double().cpu().numpy()[rec], jp[a].double().cpu().numpy())


def test_sync_rhs_chunks_and_tune(case):
    """Right-hand-side column chunks and switching schedules on a built tangent leave the
    result unchanged (bitwise)."""
    g, Ts, s, srcs, _ = case("table3-41x41x25")
    S, N, R = len(srcs), g.N, 64
    qd = torch.tensor(np.random.default_rng(11).standard_normal((S, N, R)), device=DEV, dtype=torch.float32)
    tan = _tangent(g, Ts, s, srcs)
    full = tan.solve(qd)
    tan.tune(rhs_chunk=16)
    chunked = tan.solve(qd)
    tan.tune(rhs_chunk=0, schedule=eik.SCHED_PERSISTENT)
    pers = tan.solve(qd)
    tan.tune(schedule=eik.SCHED_SYNC)
    again = tan.solve(qd)
    tan.status()
    assert torch.equal(full, chunked) and torch.equal(full, pers) and torch.equal(full, again)


def test_sync_refuses_the_lu_tier(case):
    """Blocks are applied by their inverse in this schedule: a tangent tuned to send blocks
    to the LU substitution tier is refused with a message, not run another way."""
    g, Ts, s, srcs, _ = case("cyclic-13x13x9")
    tan = _tangent(g, Ts, s, srcs)
    tan.tune(block_lu_min=2)
    q = torch.zeros((len(srcs), g.N, 4), device=DEV)
    with pytest.raises(eik.EikError) as e:
        tan.solve(q)
    assert "block_lu_min" in str(e.value)


def test_sync_stress_grid_blocks(oracle_mod):
    """The 101x101x51 steep-hill grid (slopes to 55 degrees), whose condensation holds many
    and larger SCC blocks, several per level: J p and J^T y of three sources against the
    oracle in FP32 and equal to the persistent schedule bit for bit."""
    wl = W.config5_grid(0)
    g = wl.grid
    src = wl.src[[0, 13, 31]]
    dg = eik.DeviceGrid(g)
    s = torch.tensor(wl.s, device=DEV)
    T, _ = eik.eik_forward(dg, s, src)
    tan = eik.Tangent(dg, T, s, src, rec=wl.rec, opts=eik.default_opts(schedule=eik.SCHED_SYNC))
    ref = eik.Tangent(dg, T, s, src, rec=wl.rec)
    assert max(tan.stats(a)["largest"] for a in range(len(src))) > 8
    rng = np.random.default_rng(5)
    p = torch.tensor(rng.standard_normal((g.N, wl.R)), device=DEV, dtype=torch.float32)
    y = torch.tensor(rng.standard_normal((len(src), len(wl.rec), wl.R)), device=DEV, dtype=torch.float32)
    _, jp = tan.apply(p, shared_model=True)
    gt, _ = tan.apply_T(y, sum_sources=True)
    _, jp_ref = ref.apply(p, shared_model=True)
    gt_ref, _ = ref.apply_T(y, sum_sources=True)
    tan.status()
    assert torch.equal(jp, jp_ref) and torch.equal(gt, gt_ref)
    Tn = T.cpu().numpy()
    _, G, _ = oracle_mod.metric(g)
    otans = [oracle_mod.build_tangent(g, G, Tn[a], wl.s, int(src[a])) for a in range(len(src))]
    pn, yn = p.double().cpu().numpy(), y.double().cpu().numpy()
    assert rel_err(jp.double().cpu().numpy(), oracle_mod.J(otans, wl.s, wl.rec, pn)) <= 1e-5
    assert rel_err(gt.double().cpu().numpy(), oracle_mod.JT(otans, wl.s, wl.rec, yn)) <= 1e-5


def test_sync_barrier_timeout_reported_and_context_survives(case):
    """A grid barrier that cannot complete (a test hold makes one CTA skip its arrival) ends
    every CTA's bounded wait with EIK_ERR_TIMEOUT; the next traversal on the same context is
    correct again."""
    g, Ts, s, srcs, _ = case("table3-41x41x25")
    tan = _tangent(g, Ts, s, srcs, wait_timeout_s=0.25)
    q = torch.randn((len(srcs), g.N, 2), device=DEV, dtype=torch.float64)
    good = tan.solve(q).clone()
    tan.status()
    tan.debug_hold(0, 3)
    tan.solve(q)
    with pytest.raises(eik.EikError) as e:
        tan.status()
    assert e.value.code == -5
    tan.debug_hold(-1, -1)
    again = tan.solve(q)
    tan.status()
    assert torch.equal(again, good)
