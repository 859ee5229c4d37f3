"""GPU: split_dirs gives the transpose direction its own launch state, so J p and J^T y on
one tangent run concurrently on two streams; the results equal the sequential calls bit
for bit (persistent and cluster schedules, FP32 and FP64, column chunks, node and point
sources), and the option can be switched on after the build."""
import numpy as np
import pytest
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def case():
    g = W.graph_grid((31, 31, 17), 500.0)
    srcs = np.array([g.index(5, 5, 0), g.index(25, 10, 0), g.index(12, 24, 0)], dtype=np.int32)
    s = W.curved_state(g, int(srcs[0]), 0.05).s
    dg = eik.DeviceGrid(g)
    sd = torch.tensor(s, device=DEV)
    T, _ = eik.eik_forward(dg, sd, srcs)
    rec = np.array([g.index(i, j, 0) for i in range(1, 31, 3) for j in range(1, 31, 3)], dtype=np.int32)
    return g, dg, sd, T, srcs, rec


def _inputs(g, S, n_rec, R, dtype, seed):
    rng = np.random.default_rng(seed)
    p = torch.tensor(rng.standard_normal((g.N, R)), device=DEV, dtype=dtype)
    y = torch.tensor(rng.standard_normal((S, n_rec, R)), device=DEV, dtype=dtype)
    return p, y


def _sequential(tan, p, y):
    _, d = tan.apply(p, shared_model=True)
    g, _ = tan.apply_T(y, sum_sources=True)
    tan.status()
    return d, g


def _concurrent(tan, p, y):
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    ev = torch.cuda.Event()
    ev.record()
    sa.wait_event(ev)
    sb.wait_event(ev)
    with torch.cuda.stream(sa):
        _, d = tan.apply(p, shared_model=True)
    with torch.cuda.stream(sb):
        g, _ = tan.apply_T(y, sum_sources=True)
    torch.cuda.synchronize()
    tan.status()
    return d, g


@pytest.mark.parametrize("schedule", [eik.SCHED_PERSISTENT, eik.SCHED_CLUSTER])
@pytest.mark.parametrize("dtype,R,chunk", [(torch.float32, 64, 0), (torch.float64, 8, 0), (torch.float32, 16, 4)])
def test_concurrent_directions_equal_sequential(case, schedule, dtype, R, chunk):
    g, dg, sd, T, srcs, rec = case
    p, y = _inputs(g, len(srcs), len(rec), R, dtype, R)
    ref = eik.Tangent(dg, T, sd, srcs, rec=rec, opts=eik.default_opts(schedule=schedule, rhs_chunk=chunk))
    d0, g0 = _sequential(ref, p, y)
    ref.free()
    tan = eik.Tangent(dg, T, sd, srcs, rec=rec,
                      opts=eik.default_opts(schedule=schedule, rhs_chunk=chunk, split_dirs=1, ctas_per_sm=2))
    for _ in range(3):
        d1, g1 = _concurrent(tan, p, y)
        assert torch.equal(d0, d1) and torch.equal(g0, g1)


def test_split_enabled_by_tune_and_point_sources(oracle_mod, case):
    g, dg, sd, T, srcs, rec = case
    f = np.array([[5.3, 4.6, 0.4], [20.5, 10.25, 2.75]])
    Tp, _ = eik.eik_forward_points(dg, sd, f)
    p, y = _inputs(g, len(f), len(rec), 8, torch.float64, 3)
    tan = eik.Tangent(dg, Tp, sd, f, rec=rec, points=True)
    d0, g0 = _sequential(tan, p, y)
    tan.tune(split_dirs=1, ctas_per_sm=2)
    d1, g1 = _concurrent(tan, p, y)
    assert torch.equal(d0, d1) and torch.equal(g0, g1)
