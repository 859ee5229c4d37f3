"""GPU: tangents built with items above 64 positions (eik_opts.chunk up to 256, the form for
few right-hand sides) give the same J p and J^T y bit for bit as the default items, in the
persistent schedule (the large-item kernel instance, one or two items held per CTA) and the
cluster schedule; the per-level schedules refuse them with EIK_ERR_INVALID."""
import numpy as np
import pytest
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def case():
    wl = W.config5_grid(0)
    src = wl.src[[0, 13, 31]]
    dg = eik.DeviceGrid(wl.grid)
    sd = torch.tensor(wl.s, device=DEV)
    T, _ = eik.eik_forward(dg, sd, src)
    return wl.grid, dg, sd, T, src, wl.rec


def _run(case, chunk, dtype, R, **opts):
    g, dg, sd, T, src, rec = case
    tan = eik.Tangent(dg, T, sd, src, rec=rec, opts=eik.default_opts(chunk=chunk, **opts))
    rng = np.random.default_rng(R)
    p = torch.tensor(rng.standard_normal((g.N, R)), device=DEV, dtype=dtype)
    y = torch.tensor(rng.standard_normal((len(src), len(rec), R)), device=DEV, dtype=dtype)
    dT = torch.empty((len(src), g.N, R), device=DEV, dtype=dtype)
    _, d = tan.apply(p, shared_model=True, dT_full=dT)
    gs, _ = tan.apply_T(y, sum_sources=True)
    tan.status()
    tan.free()
    return dT, d, gs


@pytest.mark.parametrize("slots", [0, 2])
@pytest.mark.parametrize("chunk", [128, 256])
@pytest.mark.parametrize("dtype,R", [(torch.float64, 1), (torch.float32, 1), (torch.float64, 4), (torch.float32, 16)])
def test_large_items_equal_default_items(case, chunk, dtype, R, slots):
    ref = _run(case, 0, dtype, R)
    got = _run(case, chunk, dtype, R, item_slots=slots)
    for u, v in zip(ref, got):
        assert torch.equal(u, v)


def test_large_items_in_cluster_schedule_and_refused_per_level(case):
    ref = _run(case, 0, torch.float64, 2)
    got = _run(case, 256, torch.float64, 2, schedule=eik.SCHED_CLUSTER)
    for u, v in zip(ref, got):
        assert torch.equal(u, v)
    with pytest.raises(eik.EikError) as e:
        _run(case, 256, torch.float64, 2, schedule=eik.SCHED_LEVELS)
    assert e.value.code == -1
