"""GPU parity at the benchmark's full size (101 x 101 x 51, 25 sources, R = 64, persistent
schedule, FP32 substitution with FP64 blocks), in the launch configuration bench.py times.

Every one of the 25 sources is compared output by output with the oracle: the oracle
solves each state itself (CPU sweeping, in a spawn-context process pool), the device
builds one tangent from those 25 oracle states, and structure (bit for bit), J p at the
receivers and each source's J_a^T y_a over all nodes are compared.  All sources are
also checked by properties that hold at any size: the scaling identity dT = -T for
dv = v (Sec. 3.2) and the adjoint pairing (Sec. 4.4)."""
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


@pytest.fixture(scope="module")
def every_source():
    """Oracle states, structure and J / J^T columns of all 25 sources (process pool)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    wl = W.config3()
    R = 64
    rng = np.random.default_rng(25)
    p = rng.standard_normal((wl.grid.N, R)).astype(np.float32)
    y = rng.standard_normal((len(wl.src), len(wl.rec), R)).astype(np.float32)
    cols = [0, 17, 40, 63]
    from tests._oracle_pool import source_reference
    pc = p[:, cols].astype(np.float64)
    jobs = [(a, pc, y[a][:, cols].astype(np.float64)) for a in range(len(wl.src))]
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1), mp_context=mp.get_context("spawn")) as ex:
        res = sorted(ex.map(source_reference, jobs), key=lambda r: r[0])
    return wl, p, y, cols, res


def test_fullsize_every_source_matches_oracle(every_source):
    """All 25 sources, FP32 with FP64 blocks (the benchmark path): structure bit for bit,
    J p at the receivers and J_a^T y_a over all nodes within 1e-5 of the oracle."""
    wl, p, y, cols, res = every_source
    g = wl.grid
    dg = eik.DeviceGrid(g)
    Ts = np.stack([r[1] for r in res])
    tan = eik.Tangent(dg, torch.tensor(Ts, device=DEV), torch.tensor(wl.s, device=DEV), wl.src, rec=wl.rec)
    for a, r in enumerate(res):
        ex = tan.export(a)
        assert np.array_equal(ex["label"], r[2]) and np.array_equal(ex["perm"], r[3]), a
        assert np.array_equal(ex["level_ptr"], r[4]), a
    pd = torch.tensor(p, device=DEV)
    yd = torch.tensor(y, device=DEV)
    _, drec = tan.apply(pd, shared_model=True)
    ga, _ = tan.apply_T(yd, sum_sources=False)
    tan.status()
    drec = drec[:, :, cols].double().cpu().numpy()
    ga = ga[:, :, cols].double().cpu().numpy()
    worst_j = worst_t = 0.0
    for a, r in enumerate(res):
        ej = np.max(np.abs(drec[a] - r[5])) / np.max(np.abs(r[5]))
        et = np.max(np.abs(ga[a] - r[6])) / np.max(np.abs(r[6]))
        worst_j, worst_t = max(worst_j, ej), max(worst_t, et)
        assert ej <= 1e-5 and et <= 1e-5, (a, ej, et)
    print(f"25 sources: worst J rel err {worst_j:.2e}, worst J^T rel err {worst_t:.2e}")


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
