"""GPU: several tangents (different grids, source counts, depths and right-hand-side
counts) traversed in one launch -- of the persistent schedule (a merged step-major item
order, several items held per CTA) by default, of the cluster schedule when the first
tangent asks for it -- give exactly what each tangent gives on its own, and match the CPU
oracle."""
import numpy as np
import pytest
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _graph(n, A, eps, srcs, every):
    g = W.graph_grid(n, A)
    Ts = np.stack([W.curved_state(g, g.index(a, b, 0), eps).T for (a, b) in srcs])
    s = W.curved_state(g, g.index(*srcs[0], 0), eps).s
    rec = np.array([g.index(i, j, 0) for i in range(0, n[0], every) for j in range(0, n[1], every)], dtype=np.int32)
    return g, Ts, s, np.array([g.index(a, b, 0) for (a, b) in srcs], dtype=np.int32), rec


def _config1():
    wl = W.config1()
    g = wl.grid
    srcs = np.array([int(wl.src[0]), g.index(45, 0)], dtype=np.int32)
    s = 1.0 / (1.5 + 0.5 * g.xyz[:, 1])
    Ts = np.stack([W.linear_velocity_T(g.xyz, g.xyz[k], 1.5, 0.5) for k in srcs])
    return g, Ts, s, srcs, np.asarray(wl.rec, dtype=np.int32)


CASES = [lambda: _graph((21, 21, 13), 500.0, 0.05, [(5, 5), (10, 10), (15, 4)], 3),
         lambda: _graph((13, 13, 9), 600.0, 0.08, [(3, 3), (6, 6)], 2),
         _config1]


@pytest.fixture(scope="module")
def setup(oracle_mod):
    out = []
    for make in CASES:
        g, Ts, s, srcs, rec = make()
        _, G, _ = oracle_mod.metric(g)
        ot = [oracle_mod.build_tangent(g, G, Ts[a], s, int(srcs[a])) for a in range(len(srcs))]
        tan = eik.Tangent(eik.DeviceGrid(g), torch.tensor(Ts, device=DEV), torch.tensor(s, device=DEV), srcs, rec=rec)
        out.append((g, s, srcs, rec, ot, tan))
    return out


@pytest.mark.parametrize("schedule", ["persistent", "cluster"])
@pytest.mark.parametrize("dtype,Rs", [(torch.float64, (2, 3, 1)), (torch.float32, (8, 16, 4)), (torch.float32, (64, 8, 32))])
def test_batch_equals_single_and_oracle(oracle_mod, setup, dtype, Rs, schedule):
    rng = np.random.default_rng(sum(Rs))
    tans = [c[-1] for c in setup]
    ps = [torch.tensor(rng.standard_normal((c[0].N, R)), device=DEV, dtype=dtype) for c, R in zip(setup, Rs)]
    ys = [torch.tensor(rng.standard_normal((len(c[2]), len(c[3]), R)), device=DEV, dtype=dtype) for c, R in zip(setup, Rs)]
    tans[0].tune(schedule=eik.SCHED_CLUSTER if schedule == "cluster" else eik.SCHED_PERSISTENT)
    jp = eik.apply_batch(tans, ps)
    jt = eik.apply_T_batch(tans, ys)
    tans[0].tune(schedule=eik.SCHED_PERSISTENT)
    tol = 1e-10 if dtype == torch.float64 else 1e-5
    for (g, s, srcs, rec, ot, tan), p, y, a, b in zip(setup, ps, ys, jp, jt):
        _, single = tan.apply(p, shared_model=True)
        gs, _ = tan.apply_T(y, sum_sources=True)
        tan.status()
        assert torch.equal(a, single)
        assert torch.equal(b, gs)
        ref = oracle_mod.J(ot, s, rec, p.double().cpu().numpy())
        assert np.max(np.abs(a.double().cpu().numpy() - ref)) <= tol * np.max(np.abs(ref))
        ref = oracle_mod.JT(ot, s, rec, y.double().cpu().numpy())
        assert np.max(np.abs(b.double().cpu().numpy() - ref)) <= tol * np.max(np.abs(ref))


def test_batch_rejects_bad_arguments(setup):
    tans = [c[-1] for c in setup]
    p = torch.zeros((setup[0][0].N, 4), device=DEV)
    with pytest.raises(ValueError):
        eik.apply_batch(tans * 2, [p] * 6)


def test_batch_rejects_a_repeated_tangent(setup):
    """Each tangent keeps its own counters: the same tangent twice in one batch is refused."""
    tans = [c[-1] for c in setup]
    ps = [torch.zeros((setup[0][0].N, 4), device=DEV)] * 2
    with pytest.raises(eik.EikError):
        eik.apply_batch([tans[0], tans[0]], ps)
