"""GPU parity at the benchmark's full size (101 x 101 x 51, 25 sources, R = 64, persistent
schedule, FP32 substitution with FP64 blocks), in the launch configuration bench.py times.

Two sources are compared output by output with the oracle: the oracle solves their
states itself (CPU sweeping), the device builds its tangent from those oracle states,
and structure (bit for bit), J p at the receivers and J^T y are compared over all
nodes.  All 25 sources are checked by properties that hold at any size: the scaling
identity dT = -T for dv = v (Sec. 3.2) and the adjoint pairing (Sec. 4.4)."""
import numpy as np
import pytest
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def full():
    wl = W.config3()
    dg = eik.DeviceGrid(wl.grid)
    s = torch.tensor(wl.s, device=DEV)
    T, cyc = eik.eik_forward(dg, s, wl.src)
    tan = eik.Tangent(dg, T, s, wl.src, rec=wl.rec)
    return wl, dg, s, T, tan


@pytest.fixture(scope="module")
def sampled(oracle_mod):
    wl = W.config3()
    g = wl.grid
    _, G, _ = oracle_mod.metric(g)
    picks = [0, 12]
    Ts, otans = [], []
    for a in picks:
        T, cyc = oracle_mod.eik_forward(g, wl.s, int(wl.src[a]))
        assert cyc > 0
        Ts.append(T)
        otans.append(oracle_mod.build_tangent(g, G, T, wl.s, int(wl.src[a])))
    return wl, picks, np.stack(Ts), otans


def test_fullsize_state_matches_oracle(full, sampled):
    wl, dg, s, T, tan = full
    _, picks, Ts, _ = sampled
    for k, a in enumerate(picks):
        t = T[a].cpu().numpy()
        assert np.max(np.abs(t - Ts[k])) <= 1e-12 * Ts[k].max()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_fullsize_sampled_sources_match_oracle(oracle_mod, sampled, dtype):
    wl, picks, Ts, otans = sampled
    g = wl.grid
    dg = eik.DeviceGrid(g)
    srcs = wl.src[picks]
    tan = eik.Tangent(dg, torch.tensor(Ts, device=DEV), torch.tensor(wl.s, device=DEV), srcs, rec=wl.rec)
    for k, ot in enumerate(otans):
        ex = tan.export(k)
        assert np.array_equal(ex["label"], ot.label) and np.array_equal(ex["perm"], ot.perm)
        assert np.array_equal(ex["level_ptr"], ot.level_ptr) and np.array_equal(ex["col"], ot.col)
    R = 64
    gen = torch.Generator(DEV).manual_seed(5)
    p = torch.randn((g.N, R), device=DEV, dtype=dtype, generator=gen)
    y = torch.randn((len(srcs), len(wl.rec), R), device=DEV, dtype=dtype, generator=gen)
    _, drec = tan.apply(p, shared_model=True)
    gsum, _ = tan.apply_T(y, sum_sources=True)
    tan.status()
    tol = 1e-5 if dtype == torch.float32 else 1e-10
    ref = oracle_mod.J(otans, wl.s, wl.rec, p.double().cpu().numpy())
    assert np.max(np.abs(drec.double().cpu().numpy() - ref)) <= tol * np.max(np.abs(ref))
    refT = oracle_mod.JT(otans, wl.s, wl.rec, y.double().cpu().numpy())
    assert np.max(np.abs(gsum.double().cpu().numpy() - refT)) <= tol * np.max(np.abs(refT))


def test_fullsize_scaling_identity_all_sources(full):
    """dv = v, i.e. ds = -s with the slowness model, gives dT = -T exactly (Sec. 3.2)."""
    wl, dg, s, T, tan = full
    p = (-s).unsqueeze(1).contiguous()
    dT = torch.empty((len(wl.src), wl.grid.N, 1), device=DEV, dtype=torch.float64)
    tan.apply(p, shared_model=True, dT_full=dT)
    tan.status()
    err = (dT[..., 0] + T).abs().max() / T.abs().max()
    assert float(err) <= 1e-12
    p32 = p.float()
    dT32 = torch.empty_like(dT, dtype=torch.float32)
    tan.apply(p32, shared_model=True, dT_full=dT32)
    err32 = (dT32[..., 0].double() + T).abs().max() / T.abs().max()
    assert float(err32) <= 1e-5


def test_fullsize_adjoint_pairing_all_sources(full):
    wl, dg, s, T, tan = full
    gen = torch.Generator(DEV).manual_seed(9)
    p = torch.randn((wl.grid.N, 2), device=DEV, dtype=torch.float64, generator=gen)
    y = torch.randn((len(wl.src), len(wl.rec), 2), device=DEV, dtype=torch.float64, generator=gen)
    _, jp = tan.apply(p, shared_model=True)
    jty, _ = tan.apply_T(y, sum_sources=True)
    l1, l2 = float((jp * y).sum()), float((p * jty).sum())
    assert abs(l1 - l2) <= 1e-13 * max(abs(l1), abs(l2))
