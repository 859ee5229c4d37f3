"""GPU parity of the multi-slot persistent schedule (item_slots 2..4: every CTA holds
several work items and computes whichever has its upstream items done first): bit-for-bit
equality with the single-slot persistent schedule (the same per-node arithmetic), the
Jacobian actions against the CPU FP64 oracle, and the bounded wait's time-out."""
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


@pytest.fixture(scope="module")
def table3():
    return _graph_case((41, 41, 25), 500.0, 0.05, [(10, 10), (20, 20), (30, 10)])


def _tangent(g, Ts, s, srcs, rec=None, **kw):
    return eik.Tangent(eik.DeviceGrid(g), torch.tensor(Ts, device=DEV), torch.tensor(s, device=DEV), srcs,
                       rec=rec, opts=eik.default_opts(**kw))


@pytest.mark.parametrize("slots", [2, 3, 4])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("deps", [1, 0])
def test_multi_matches_single_slot_bitwise(table3, slots, dtype, deps):
    """A^-1 q and A^-T r with 2..4 items held per CTA, per-item or whole-level waits, equal
    the single-slot persistent schedule bit for bit (the cases hold nontrivial blocks)."""
    g, Ts, s, srcs = table3
    S, N, R = len(srcs), g.N, 64
    qd = torch.tensor(np.random.default_rng(17).standard_normal((S, N, R)), device=DEV, dtype=dtype)
    ref = _tangent(g, Ts, s, srcs, item_deps=deps)
    rx, rl = ref.solve(qd), ref.solve_T(qd)
    tan = _tangent(g, Ts, s, srcs, item_deps=deps)
    tan.tune(item_slots=slots)
    x, lam = tan.solve(qd), tan.solve_T(qd)
    tan.status()
    assert sum(tan.stats(a)["nontrivial"] for a in range(S)) > 0
    assert torch.equal(x, rx) and torch.equal(lam, rl)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_multi_jacobian_actions_against_oracle(oracle_mod, dtype):
    """J p and J^T y (Sec. 4.4) with four items per CTA against the oracle."""
    g, Ts, s, srcs = _graph_case((13, 13, 9), 600.0, 0.08, [(3, 3), (6, 6), (9, 3)])
    _, G, _ = oracle_mod.metric(g)
    otans = [oracle_mod.build_tangent(g, G, Ts[a], s, int(srcs[a])) for a in range(len(srcs))]
    rec = np.array([g.index(i, j, 0) for i in range(0, 13, 2) for j in range(0, 13, 3)], dtype=np.int32)
    tan = _tangent(g, Ts, s, srcs, rec=rec)
    tan.tune(item_slots=4)
    S, N, R = len(srcs), g.N, 8
    rng = np.random.default_rng(3)
    p = torch.tensor(rng.standard_normal((N, R)), device=DEV, dtype=dtype)
    y = torch.tensor(rng.standard_normal((S, len(rec), R)), device=DEV, dtype=dtype)
    _, jp = tan.apply(p, shared_model=True)
    gs, _ = tan.apply_T(y, sum_sources=True)
    tan.status()
    pp, yy = p.double().cpu().numpy(), y.double().cpu().numpy()
    assert rel_err(jp.double().cpu().numpy(), oracle_mod.J(otans, s, rec, pp)) <= TOL[dtype]
    assert rel_err(gs.double().cpu().numpy(), oracle_mod.JT(otans, s, rec, yy)) <= TOL[dtype]


def test_multi_wait_timeout_reported_and_context_survives(table3):
    """A wait that can never be satisfied (a held level count) ends with EIK_ERR_TIMEOUT in
    bounded time; the next traversal on the same context is correct again."""
    g, Ts, s, srcs = table3
    tan = _tangent(g, Ts, s, srcs, wait_timeout_s=0.25)
    tan.tune(item_slots=4, wait_timeout_s=0.25)
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
