"""GPU: the node <- cell map of a cell-based velocity model and the Jacobian actions on
cells it gives (J A p, A^T J^T y), through the C ABI, against the oracle."""
import numpy as np
import pytest
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _grids():
    g3 = W.graph_grid((21, 21, 13), 500.0)
    wl = W.config1()
    return [g3, wl.grid]


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_cell_map_against_oracle(oracle_mod, which, dtype):
    g = _grids()[which]
    A = oracle_mod.cell_average(g)
    dg = eik.DeviceGrid(g)
    rng = np.random.default_rng(3)
    pc = torch.tensor(rng.standard_normal((A.shape[1], 5)), device=DEV, dtype=dtype)
    gn = torch.tensor(rng.standard_normal((g.N, 5)), device=DEV, dtype=dtype)
    pn = eik.cells_to_nodes(dg, pc)
    gc = eik.nodes_to_cells(dg, gn)
    torch.cuda.synchronize()
    tol = 1e-14 if dtype == torch.float64 else 1e-6
    ref_n = A @ pc.double().cpu().numpy()
    ref_c = A.T @ gn.double().cpu().numpy()
    assert np.max(np.abs(pn.double().cpu().numpy() - ref_n)) <= tol * np.max(np.abs(ref_n))
    assert np.max(np.abs(gc.double().cpu().numpy() - ref_c)) <= tol * np.max(np.abs(ref_c))


def test_jacobian_on_cells(oracle_mod):
    """J_cells p = J (A p) and J_cells^T y = A^T J^T y for a velocity model on cells
    (3 sources, 3-D), and the pairing <J_cells p, y> = <p, J_cells^T y>."""
    g = W.graph_grid((21, 21, 13), 500.0)
    srcs = np.array([g.index(5, 5, 0), g.index(15, 10, 0), g.index(10, 16, 0)], dtype=np.int32)
    Ts = np.stack([W.curved_state(g, int(k), 0.05).T for k in srcs])
    s = W.curved_state(g, int(srcs[0]), 0.05).s
    rec = np.array([g.index(i, j, 0) for i in range(1, 21, 3) for j in range(1, 21, 3)], dtype=np.int32)
    _, G, _ = oracle_mod.metric(g)
    otans = [oracle_mod.build_tangent(g, G, Ts[a], s, int(srcs[a])) for a in range(len(srcs))]
    dg = eik.DeviceGrid(g)
    tan = eik.Tangent(dg, torch.tensor(Ts, device=DEV), torch.tensor(s, device=DEV), srcs, rec=rec,
                      opts=eik.default_opts(model=eik.MODEL_VELOCITY))
    A = oracle_mod.cell_average(g)
    rng = np.random.default_rng(4)
    pc = torch.tensor(rng.standard_normal((A.shape[1], 4)), device=DEV)
    y = torch.tensor(rng.standard_normal((len(srcs), len(rec), 4)), device=DEV)
    _, d = tan.apply(eik.cells_to_nodes(dg, pc), shared_model=True)
    gnode, _ = tan.apply_T(y, sum_sources=True)
    gc = eik.nodes_to_cells(dg, gnode)
    tan.status()
    ref_d = oracle_mod.J(otans, s, rec, A @ pc.cpu().numpy(), model=oracle_mod.MODEL_VELOCITY)
    ref_g = A.T @ oracle_mod.JT(otans, s, rec, y.cpu().numpy(), model=oracle_mod.MODEL_VELOCITY)
    assert np.max(np.abs(d.cpu().numpy() - ref_d)) <= 1e-10 * np.max(np.abs(ref_d))
    assert np.max(np.abs(gc.cpu().numpy() - ref_g)) <= 1e-10 * np.max(np.abs(ref_g))
    l1, l2 = float((d * y).sum()), float((pc * gc).sum())
    assert abs(l1 - l2) <= 1e-12 * max(abs(l1), abs(l2))
