"""GPU: a grid with more than 2^22 nodes (the canonical-order sort key sizes its node and
component fields to the grid), structure bit for bit and J, J^T against the oracle."""
import numpy as np
import pytest
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def test_grid_beyond_2_pow_22_nodes(oracle_mod):
    g = W.graph_grid((163, 163, 160), 300.0)
    assert g.N > (1 << 22)
    src = np.array([W.quarter_source(g)], dtype=np.int32)
    st = W.curved_state(g, int(src[0]), 0.05)
    dg = eik.DeviceGrid(g)
    tan = eik.Tangent(dg, torch.tensor(st.T[None], device=DEV), torch.tensor(st.s, device=DEV), src,
                      rec=np.array([g.index(i, j, 0) for i in range(0, 163, 9) for j in range(0, 163, 9)],
                                   dtype=np.int32))
    _, G, _ = oracle_mod.metric(g)
    ot = oracle_mod.build_tangent(g, G, st.T, st.s, int(src[0]))
    ex = tan.export(0)
    assert np.array_equal(ex["label"], ot.label) and np.array_equal(ex["perm"], ot.perm)
    assert np.array_equal(ex["level_ptr"], ot.level_ptr)
    rng = np.random.default_rng(17)
    q = torch.tensor(rng.standard_normal((1, g.N, 2)), device=DEV)
    x = tan.solve(q)
    lam = tan.solve_T(q)
    tan.status()
    qn = q.cpu().numpy()[0]
    ref = oracle_mod.solve(ot, qn)
    assert np.max(np.abs(x.cpu().numpy()[0] - ref)) <= 1e-10 * np.max(np.abs(ref))
    ref = oracle_mod.solve_T(ot, qn)
    assert np.max(np.abs(lam.cpu().numpy()[0] - ref)) <= 1e-10 * np.max(np.abs(ref))
