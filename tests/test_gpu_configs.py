"""GPU parity on the 2-D benchmark configurations at their full sizes (every source,
every right-hand side, every output), with states solved by the oracle itself."""
import numpy as np
import pytest
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _oracle_states(O, wl):
    g = wl.grid
    _, G, _ = O.metric(g)
    Ts, tans = [], []
    for k in wl.src:
        T, cyc = O.eik_forward(g, wl.s, int(k))
        assert cyc > 0
        Ts.append(T)
        tans.append(O.build_tangent(g, G, T, wl.s, int(k)))
    return np.stack(Ts), tans


@pytest.mark.parametrize("cfg", ["config1", "config2"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_config_full_parity(oracle_mod, cfg, dtype):
    wl = getattr(W, cfg)()
    g = wl.grid
    Ts, otans = _oracle_states(oracle_mod, wl)
    dg = eik.DeviceGrid(g)
    # the device state solve reaches the same fixed point
    Td, _ = eik.eik_forward(dg, torch.tensor(wl.s, device=DEV), wl.src)
    assert np.max(np.abs(Td.cpu().numpy() - Ts)) <= 1e-12 * Ts.max()
    tan = eik.Tangent(dg, torch.tensor(Ts, device=DEV), torch.tensor(wl.s, device=DEV), wl.src, rec=wl.rec)
    for a, ot in enumerate(otans):
        ex = tan.export(a)
        assert np.array_equal(ex["label"], ot.label) and np.array_equal(ex["perm"], ot.perm)
        assert np.array_equal(ex["level_ptr"], ot.level_ptr)
    S, N, R = wl.S, g.N, wl.R
    rng = np.random.default_rng(wl.seed)
    p = torch.tensor(rng.standard_normal((S, N, R)), device=DEV, dtype=dtype)
    y = torch.tensor(rng.standard_normal((S, len(wl.rec), R)), device=DEV, dtype=dtype)
    dT = torch.empty_like(p)
    _, drec = tan.apply(p, shared_model=False, dT_full=dT)
    gS, _ = tan.apply_T(y, sum_sources=False)
    tan.status()
    tol = 1e-5 if dtype == torch.float32 else 1e-10
    pn, yn = p.double().cpu().numpy(), y.double().cpu().numpy()
    for a, ot in enumerate(otans):
        q = ot.cs[:, None] * pn[a]
        ref = oracle_mod.solve(ot, q)
        assert np.max(np.abs(dT[a].double().cpu().numpy() - ref)) <= tol * np.max(np.abs(ref))
    refJ = oracle_mod.J(otans, wl.s, wl.rec, pn, shared=False)
    assert np.max(np.abs(drec.double().cpu().numpy() - refJ)) <= tol * np.max(np.abs(refJ))
    refT = oracle_mod.JT(otans, wl.s, wl.rec, yn, sum_sources=False)
    assert np.max(np.abs(gS.double().cpu().numpy() - refT)) <= tol * np.max(np.abs(refT))
