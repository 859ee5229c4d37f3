"""GPU: off-grid receivers (multilinear P in J and J^T) through the C ABI against the
oracle; node positions reproduce the on-grid path; chunked right-hand sides agree with
one pass; coordinates outside the grid are refused."""
import numpy as np
import pytest
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _case(oracle_mod, opts=None, rec=None):
    g = W.graph_grid((21, 21, 13), 500.0)
    srcs = np.array([g.index(5, 5, 0), g.index(15, 10, 0), g.index(10, 16, 0)], dtype=np.int32)
    Ts = np.stack([W.curved_state(g, int(k), 0.05).T for k in srcs])
    s = W.curved_state(g, int(srcs[0]), 0.05).s
    _, G, _ = oracle_mod.metric(g)
    otans = [oracle_mod.build_tangent(g, G, Ts[a], s, int(srcs[a])) for a in range(len(srcs))]
    tan = eik.Tangent(eik.DeviceGrid(g), torch.tensor(Ts, device=DEV), torch.tensor(s, device=DEV), srcs, rec=rec,
                      opts=opts)
    return g, s, srcs, otans, tan


def _positions(g, S, n, seed):
    rng = np.random.default_rng(seed)
    f = np.empty((S, n, 3))
    f[:, :, 0] = rng.uniform(0, g.n[0] - 1, (S, n))
    f[:, :, 1] = rng.uniform(0, g.n[1] - 1, (S, n))
    f[:, :, 2] = rng.choice([0.0, 0.5, 3.25, g.n[2] - 1.0], (S, n))
    return f


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_interp_receivers_against_oracle(oracle_mod, dtype):
    g, s, srcs, otans, tan = _case(oracle_mod)
    f = _positions(g, len(srcs), 30, 11)
    tan.set_receivers(f)
    Ps = [oracle_mod.receiver_interp(g, f[a]) for a in range(len(srcs))]
    rng = np.random.default_rng(12)
    p = torch.tensor(rng.standard_normal((g.N, 8)), device=DEV, dtype=dtype)
    y = torch.tensor(rng.standard_normal((len(srcs), 30, 8)), device=DEV, dtype=dtype)
    d = tan.apply_interp(p)
    gg = tan.apply_interp_T(y)
    tan.status()
    tol = 1e-10 if dtype == torch.float64 else 1e-5
    ref_d = oracle_mod.J_interp(otans, s, Ps, p.double().cpu().numpy())
    ref_g = oracle_mod.JT_interp(otans, s, Ps, y.double().cpu().numpy())
    assert np.max(np.abs(d.double().cpu().numpy() - ref_d)) <= tol * np.max(np.abs(ref_d))
    assert np.max(np.abs(gg.double().cpu().numpy() - ref_g)) <= tol * np.max(np.abs(ref_g))


def test_interp_on_nodes_equals_on_grid_path_and_chunking(oracle_mod):
    g0 = W.graph_grid((21, 21, 13), 500.0)
    rec = np.array([g0.index(i, j, 0) for i in range(1, 21, 3) for j in range(1, 21, 3)], dtype=np.int32)
    g, s, srcs, otans, tan = _case(oracle_mod, rec=rec)
    ijk = np.array([[i, j, 0] for i in range(1, 21, 3) for j in range(1, 21, 3)], dtype=np.float64)
    tan.set_receivers(np.repeat(ijk[None], len(srcs), axis=0))
    rng = np.random.default_rng(13)
    p = torch.tensor(rng.standard_normal((g.N, 12)), device=DEV)
    y = torch.tensor(rng.standard_normal((len(srcs), len(rec), 12)), device=DEV)
    _, d_grid = tan.apply(p, shared_model=True)
    g_grid, _ = tan.apply_T(y, sum_sources=True)
    d = tan.apply_interp(p)
    gg = tan.apply_interp_T(y)
    assert float((d - d_grid).abs().max()) <= 1e-14 * float(d_grid.abs().max())
    assert float((gg - g_grid).abs().max()) <= 1e-14 * float(g_grid.abs().max())
    tan.tune(rhs_chunk=4)
    assert torch.equal(tan.apply_interp(p), d)
    assert torch.equal(tan.apply_interp_T(y), gg)
    tan.status()
    with pytest.raises(eik.EikError) as e:
        tan.set_receivers(np.full((len(srcs), 1, 3), 25.0))
    assert e.value.code == -1
