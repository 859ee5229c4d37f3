"""GPU parity on the steep-hill stress grids (slopes up to about 55 deg): sampled sources at
full grid size against the oracle (which builds its tangents from the same states), and
right-hand-side chunking on the largest grid, where one [S][N][R] field would be 134 GB
for all 64 sources at R = 128."""
import numpy as np
import pytest
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _sampled(oracle_mod, which, pick, fp32_state=False):
    wl = W.config5_grid(which)
    g = wl.grid
    src = wl.src[list(pick)]
    dg = eik.DeviceGrid(g)
    s = torch.tensor(wl.s, device=DEV)
    T, _ = eik.eik_forward(dg, s, src, opts=eik.default_opts(eik_fp32=int(fp32_state)))
    Tn = T.cpu().numpy()
    _, G, _ = oracle_mod.metric(g)
    otans = [oracle_mod.build_tangent(g, G, Tn[a], wl.s, int(src[a])) for a in range(len(src))]
    return wl, g, dg, s, T, src, otans


def _rel(a, b):
    return float(np.max(np.abs(a.double().cpu().numpy() - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_stress_grid0_sampled_sources(oracle_mod, dtype):
    """101x101x51 steep-hill grid, 3 of its 32 sources, R = 8: structure bit for bit, then
    J p (shared model) and J^T y (summed) against the oracle."""
    wl, g, dg, s, T, src, otans = _sampled(oracle_mod, 0, (0, 13, 31))
    tan = eik.Tangent(dg, T, s, src, rec=wl.rec)
    for a, ot in enumerate(otans):
        ex = tan.export(a)
        assert np.array_equal(ex["label"], ot.label) and np.array_equal(ex["perm"], ot.perm)
        assert np.array_equal(ex["level_ptr"], ot.level_ptr)
    rng = np.random.default_rng(wl.seed)
    p = torch.tensor(rng.standard_normal((g.N, wl.R)), device=DEV, dtype=dtype)
    y = torch.tensor(rng.standard_normal((len(src), len(wl.rec), wl.R)), device=DEV, dtype=dtype)
    _, drec = tan.apply(p, shared_model=True)
    gs, _ = tan.apply_T(y, sum_sources=True)
    tan.status()
    tol = 1e-10 if dtype == torch.float64 else 1e-5
    pn, yn = p.double().cpu().numpy(), y.double().cpu().numpy()
    assert _rel(drec, oracle_mod.J(otans, wl.s, wl.rec, pn)) <= tol
    assert _rel(gs, oracle_mod.JT(otans, wl.s, wl.rec, yn)) <= tol


def test_stress_grid2_rhs_chunking(oracle_mod):
    """201x201x101 grid, 2 sources, R = 128 FP32: traversing the right-hand sides in chunks
    of 32 gives the same J p and J^T y bit for bit as one pass; four sampled columns agree
    with the oracle at full grid size."""
    wl, g, dg, s, T, src, otans = _sampled(oracle_mod, 2, (0, 45), fp32_state=True)
    R = wl.R
    rng = np.random.default_rng(wl.seed)
    p = torch.tensor(rng.standard_normal((g.N, R)), device=DEV, dtype=torch.float32)
    y = torch.tensor(rng.standard_normal((len(src), len(wl.rec), R)), device=DEV, dtype=torch.float32)
    res = {}
    for chunk in (0, 32):
        tan = eik.Tangent(dg, T, s, src, rec=wl.rec, opts=eik.default_opts(rhs_chunk=chunk))
        _, drec = tan.apply(p, shared_model=True)
        gs, _ = tan.apply_T(y, sum_sources=True)
        tan.status()
        res[chunk] = (drec, gs)
        tan.free()
    assert torch.equal(res[0][0], res[32][0]) and torch.equal(res[0][1], res[32][1])
    cols = [0, 41, 90, 127]
    pn = p[:, cols].double().cpu().numpy()
    yn = y[:, :, cols].double().cpu().numpy()
    assert _rel(res[32][0][:, :, cols], oracle_mod.J(otans, wl.s, wl.rec, pn)) <= 1e-5
    assert _rel(res[32][1][:, cols], oracle_mod.JT(otans, wl.s, wl.rec, yn)) <= 1e-5
