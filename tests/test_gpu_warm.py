"""GPU: the warm-started state solve (eik_forward_warm, the re-setup of an outer
Gauss-Newton iteration): from the converged state of the same model it stops after one
cycle with the same field; after a 1 % smooth model update it converges to the fixed point
of a cold start (and of the oracle) in fewer cycles; in place and with the FP32 far field."""
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
    s = W.curved_state(g, g.index(5, 5, 0), 0.05).s
    src = np.array([g.index(5, 5, 0), g.index(25, 10, 0), g.index(12, 24, 0)], dtype=np.int32)
    x = g.xyz
    s2 = s * (1.0 + 0.01 * np.sin(2 * np.pi * x[:, 0] / 2000.0) * np.cos(2 * np.pi * x[:, 1] / 3000.0))
    return g, s, s2, src


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


def test_warm_start_from_the_solution_stops_at_once(case):
    g, s, _, src = case
    dg = eik.DeviceGrid(g)
    sd = torch.tensor(s, device=DEV)
    T, cyc = eik.eik_forward(dg, sd, src)
    T2, cyc2 = eik.eik_forward(dg, sd, src, T_init=T)
    assert cyc > 3 and cyc2 == 1
    assert _rel(T2, T) <= 1e-12


@pytest.mark.parametrize("fp32", [0, 1])
def test_warm_start_after_a_model_update(oracle_mod, case, fp32):
    g, s, s2, src = case
    dg = eik.DeviceGrid(g)
    opts = eik.default_opts(eik_fp32=fp32)
    T, _ = eik.eik_forward(dg, torch.tensor(s, device=DEV), src, opts=opts)
    s2d = torch.tensor(s2, device=DEV)
    cold, cyc_cold = eik.eik_forward(dg, s2d, src, opts=opts)
    warm, cyc_warm = eik.eik_forward(dg, s2d, src, opts=opts, T_init=T)
    assert cyc_warm < cyc_cold
    tol = 1e-9 if not fp32 else 1e-5
    assert _rel(warm, cold) <= tol
    if not fp32:
        ref = np.stack([oracle_mod.eik_forward(g, s2, int(k))[0] for k in src])
        assert _rel(warm.cpu(), torch.tensor(ref)) <= tol
    # in place: T_init and the output are the same buffer
    buf = T.clone()
    eik.eik_forward(dg, s2d, src, opts=opts, out=buf, T_init=buf)
    assert torch.equal(buf, warm)
