"""GPU: the two small operations the binding used to do in PyTorch now run in the
library -- the accumulated source sum of J^T y over source chunks (tangent_apply_T with
sum_sources = 2) and the Gauss-Newton right-hand side [-W_d r; 0; 0] (gn_rhs) -- and
give exactly the values the plain definitions give."""
import numpy as np
import pytest
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _tangent(model=eik.MODEL_SLOWNESS):
    g = W.graph_grid((21, 21, 13), 500.0)
    srcs = np.array([g.index(5, 5, 0), g.index(15, 10, 0), g.index(10, 16, 0)], dtype=np.int32)
    Ts = np.stack([W.curved_state(g, int(k), 0.05).T for k in srcs])
    s = W.curved_state(g, int(srcs[0]), 0.05).s
    rec = np.array([g.index(i, j, 0) for i in range(1, 21, 3) for j in range(1, 21, 3)], dtype=np.int32)
    tan = eik.Tangent(eik.DeviceGrid(g), torch.tensor(Ts, device=DEV), torch.tensor(s, device=DEV), srcs, rec=rec,
                      opts=eik.default_opts(model=model))
    return g, s, srcs, rec, tan


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_apply_T_accumulates_the_source_sum(dtype):
    """g0 + sum_a J_a^T y_a, formed by the library in one call, equals g0 plus the
    separately computed sum, element for element."""
    g, s, srcs, rec, tan = _tangent()
    rng = np.random.default_rng(5)
    y = torch.tensor(rng.standard_normal((len(srcs), len(rec), 8)), device=DEV, dtype=dtype)
    g0 = torch.tensor(rng.standard_normal((g.N, 8)), device=DEV, dtype=dtype)
    ref, _ = tan.apply_T(y, sum_sources=True)
    acc = g0.clone()
    tan.apply_T(y, sum_sources=True, g=acc, accumulate=True)
    tan.status()
    assert torch.equal(acc, g0 + ref)
    with pytest.raises(ValueError):
        tan.apply_T(y, sum_sources=False, g=acc, accumulate=True)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_gn_rhs_on_the_device(dtype):
    """b = [-W_d r; 0; 0] of Eq. (augmented-ls) from gn_rhs equals the definition
    (FP64 product, then rounded to the solver's vector type)."""
    g, s, srcs, rec, tan = _tangent(eik.MODEL_VELOCITY)
    rng = np.random.default_rng(8)
    wd = torch.tensor(1.0 / (3e-4 + 3e-3 * rng.uniform(0.5, 1.5, (len(srcs), len(rec)))), device=DEV)
    r = torch.tensor(rng.standard_normal((len(srcs), len(rec))) * 1e-3, device=DEV)
    gn = eik.GN(tan, wd, torch.tensor(1.0 / s, device=DEV), 0.01, 0.1, dtype=dtype)
    b = gn.rhs(r)
    torch.cuda.synchronize()
    ref = torch.zeros(gn.n_rows, dtype=dtype, device=DEV)
    ref[:gn.n_data] = (-(wd * r)).reshape(-1).to(dtype)
    assert torch.equal(b, ref)
