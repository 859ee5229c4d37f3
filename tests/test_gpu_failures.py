"""GPU: the failure codes reach the caller as plain return values, with the context left
usable -- a singular SCC block in tangent_build (a state whose closed cyclic component
violates the local-invertibility condition of Sec. 4.2) and a state solve or sweep that
runs out of cycles.  Nothing here faults, traps or hangs the device."""
import numpy as np
import pytest
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def test_singular_block_is_reported_by_tangent_build():
    g, T, s, src = W.closed_cycle_case()
    dg = eik.DeviceGrid(g)
    with pytest.raises(eik.EikError) as e:
        eik.Tangent(dg, torch.tensor(T[None], device=DEV), torch.tensor(s, device=DEV), [src])
    assert e.value.code == -3 and "singular" in str(e.value)
    # the context is still usable: a regular state builds and solves
    wl = W.config1()
    dg1 = eik.DeviceGrid(wl.grid)
    T1 = W.linear_velocity_T(wl.grid.xyz, wl.grid.xyz[int(wl.src[0])], 1.5, 0.5)
    tan = eik.Tangent(dg1, torch.tensor(T1[None], device=DEV), torch.tensor(wl.s, device=DEV), [int(wl.src[0])])
    x = tan.solve(torch.ones((1, wl.grid.N, 1), device=DEV, dtype=torch.float64))
    tan.status()
    assert torch.isfinite(x).all()


def test_state_solve_reports_non_convergence():
    wl = W.config1()
    dg = eik.DeviceGrid(wl.grid)
    sd = torch.tensor(wl.s, device=DEV)
    with pytest.raises(eik.EikError) as e:
        eik.eik_forward(dg, sd, [int(wl.src[0])], eik.default_opts(eik_max_cycles=1))
    assert e.value.code == -4
    T, cyc = eik.eik_forward(dg, sd, [int(wl.src[0])])      # and converges with the default limit
    assert cyc > 1 and torch.isfinite(T).all()


@pytest.mark.parametrize("transpose", [False, True])
def test_sweeping_reports_non_convergence(transpose):
    g = W.graph_grid((21, 21, 13), 500.0)
    src = W.quarter_source(g)
    st = W.curved_state(g, src, 0.05)
    tan = eik.Tangent(eik.DeviceGrid(g), torch.tensor(st.T[None], device=DEV), torch.tensor(st.s, device=DEV), [src])
    b = torch.tensor(np.random.default_rng(2).standard_normal((1, g.N, 4)), device=DEV)
    with pytest.raises(eik.EikError) as e:
        tan.sweep(b, transpose=transpose, opts=eik.default_opts(sweep_max_cycles=1))
    assert e.value.code == -4
    x, cyc = tan.sweep(b, transpose=transpose)
    ref = tan.solve_T(b) if transpose else tan.solve(b)
    tan.status()
    assert cyc > 1 and float((x - ref).abs().max() / ref.abs().max()) <= 1e-10
