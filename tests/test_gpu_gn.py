"""GPU: the augmented Gauss-Newton operator K = [W_d J; lam R; lam S_k] and device LSMR
on it (Sec. 4.5), through the C ABI, against the CPU oracle."""
import numpy as np
import pytest
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _case_2d():
    wl = W.config1()
    g = wl.grid
    srcs = np.array([wl.src[0], g.index(45, 0)], dtype=np.int32)
    s = 1.0 / (1.5 + 0.5 * g.xyz[:, 1])
    Ts = np.stack([W.linear_velocity_T(g.xyz, g.xyz[k], 1.5, 0.5) for k in srcs])
    return g, Ts, s, srcs, np.asarray(wl.rec, dtype=np.int32), 0.05


def _case_3d():
    g = W.graph_grid((21, 21, 13), 500.0)
    srcs = np.array([g.index(5, 5, 0), g.index(15, 10, 0), g.index(10, 16, 0)], dtype=np.int32)
    Ts = np.stack([W.curved_state(g, int(k), 0.05).T for k in srcs])
    s = W.curved_state(g, int(srcs[0]), 0.05).s
    rec = np.array([g.index(i, j, 0) for i in range(1, 21, 3) for j in range(1, 21, 3)], dtype=np.int32)
    return g, Ts, s, srcs, rec, 0.01


def _setup(oracle_mod, case, dtype=torch.float64, gamma=1.0):
    g, Ts, s, srcs, rec, lam = case()
    _, G, _ = oracle_mod.metric(g)
    otans = [oracle_mod.build_tangent(g, G, Ts[a], s, int(srcs[a])) for a in range(len(srcs))]
    tan = eik.Tangent(eik.DeviceGrid(g), torch.tensor(Ts, device=DEV), torch.tensor(s, device=DEV), srcs, rec=rec,
                      opts=eik.default_opts(model=eik.MODEL_VELOCITY))
    rng = np.random.default_rng(31)
    wd = 1.0 / (3e-4 + 3e-3 * rng.uniform(0.5, 1.5, (len(srcs), len(rec))))
    vk = 1.0 / s
    K, KT, m = oracle_mod.gn_operator(g, otans, s, rec, wd, vk, lam, gamma, model=oracle_mod.MODEL_VELOCITY)
    gn = eik.GN(tan, torch.tensor(wd, device=DEV), torch.tensor(vk, device=DEV), lam, gamma, dtype=dtype)
    return g, tan, gn, K, KT, m, wd, rng


def _rel(a, b):
    a = a.double().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("case", [_case_2d, _case_3d])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_gn_operator_against_oracle(oracle_mod, case, dtype):
    """K p and K^T y (all three blocks, R's row layout included) against the oracle, and
    the device pairing <K p, y> = <p, K^T y>."""
    g, tan, gn, K, KT, m, wd, rng = _setup(oracle_mod, case, dtype)
    assert gn.n_rows == m
    tol = 1e-10 if dtype == torch.float64 else 1e-5
    p = torch.tensor(rng.standard_normal(g.N), device=DEV, dtype=dtype)
    y = torch.tensor(rng.standard_normal(m), device=DEV, dtype=dtype)
    Kp, KTy = gn.apply(p), gn.apply_T(y)
    tan.status()
    pr, yr = p.double().cpu().numpy(), y.double().cpu().numpy()
    e1, e2 = _rel(Kp, K(pr)), _rel(KTy, KT(yr))
    assert e1 <= tol, e1
    assert e2 <= tol, e2
    # each block separately, so a wrong block cannot hide behind a large other one
    nd, nR = gn.n_data, gn.n_rough
    ref = K(pr)
    for lo, hi in ((0, nd), (nd, nd + nR), (nd + nR, m)):
        assert _rel(Kp[lo:hi], ref[lo:hi]) <= tol
    if dtype == torch.float64:
        l1, l2 = float(Kp @ y), float(p @ KTy)
        assert abs(l1 - l2) <= 1e-12 * max(abs(l1), abs(l2))


@pytest.mark.parametrize("case", [_case_2d, _case_3d])
def test_gn_lsmr_matches_oracle(oracle_mod, case):
    """Device LSMR (FP64) against the oracle's: iterate and norms at 5 iterations; at 40
    iterations graph-replayed and eager runs are bitwise equal, and the carried |r| and
    |K^T r| are the true norms of the returned x (evaluated with the device K)."""
    g, tan, gn, K, KT, m, wd, rng = _setup(oracle_mod, case)
    r = rng.standard_normal(wd.shape) * 1e-3
    b = np.concatenate([-(wd * r).ravel(), np.zeros(m - wd.size)])
    bd = torch.tensor(b, device=DEV)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        gn.start(bd)
        gn.iterate(5, use_graph=False)
        x5, sc5 = gn.solution()
        out = {}
        for use_graph in (True, False):
            gn.start(bd)
            gn.iterate(40, use_graph=use_graph)
            out[use_graph] = gn.solution()
    stream.synchronize()
    tan.status()
    xo, info = oracle_mod.lsmr(K, KT, b, 5)
    assert _rel(x5, xo) <= 1e-9
    for k in ("normr", "normar", "norma", "normx"):
        assert abs(sc5[k] - info[k]) <= 1e-9 * abs(info[k])
    assert torch.equal(out[True][0], out[False][0])
    x40, sc40 = out[True]
    with torch.cuda.stream(stream):
        res = bd - gn.apply(x40)
        ktr = gn.apply_T(res)
    stream.synchronize()
    assert abs(sc40["normr"] - float(res.norm())) <= 1e-9 * float(bd.norm())
    assert abs(sc40["normar"] - float(ktr.norm())) <= 1e-9 * float(gn.apply_T(bd).norm())


def test_gn_lsmr_fp32_and_stopping_rule(oracle_mod):
    """FP32 LSMR follows the FP64 oracle within single-precision error at 5 iterations,
    and GN.lsmr stops once |K^T r| <= atol |K| |r|, with a residual within 1e-3 of the
    minimum the oracle's converged LSMR reaches."""
    g, tan, gn, K, KT, m, wd, rng = _setup(oracle_mod, _case_3d, dtype=torch.float32)
    r = rng.standard_normal(wd.shape) * 1e-3
    b = np.concatenate([-(wd * r).ravel(), np.zeros(m - wd.size)])
    bd = torch.tensor(b, device=DEV, dtype=torch.float32)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        gn.start(bd)
        gn.iterate(5)
        x5, _ = gn.solution()
        x, sc = gn.lsmr(bd, atol=1e-4, max_iters=400)
    stream.synchronize()
    tan.status()
    xo, _ = oracle_mod.lsmr(K, KT, b.astype(np.float32).astype(np.float64), 5)
    assert _rel(x5, xo) <= 1e-4
    assert sc["normar"] <= 1e-4 * sc["norma"] * sc["normr"]
    _, info = oracle_mod.lsmr(K, KT, b, 400)
    rx = np.linalg.norm(b - K(x.double().cpu().numpy()))
    assert abs(rx - info["normr"]) <= 1e-3 * info["normr"]


@pytest.mark.parametrize("case", [_case_2d, _case_3d])
def test_gn_on_cells_against_oracle(oracle_mod, case):
    """The operator with the model on cells (J A p, R on the cell grid, S on cell
    velocities): K p, K^T y and 5 LSMR iterations against the oracle (FP64)."""
    g, Ts, s, srcs, rec, lam = case()
    _, G, _ = oracle_mod.metric(g)
    otans = [oracle_mod.build_tangent(g, G, Ts[a], s, int(srcs[a])) for a in range(len(srcs))]
    tan = eik.Tangent(eik.DeviceGrid(g), torch.tensor(Ts, device=DEV), torch.tensor(s, device=DEV), srcs, rec=rec,
                      opts=eik.default_opts(model=eik.MODEL_VELOCITY))
    rng = np.random.default_rng(41)
    nc = oracle_mod.cell_average(g).shape[1]
    vc = 2.0 + rng.uniform(0.0, 0.5, nc)
    wd = 1.0 / (3e-4 + 3e-3 * rng.uniform(0.5, 1.5, (len(srcs), len(rec))))
    K, KT, m = oracle_mod.gn_operator(g, otans, s, rec, wd, vc, lam, 1.0, cells=True)
    gn = eik.GN(tan, torch.tensor(wd, device=DEV), torch.tensor(vc, device=DEV), lam, 1.0, cells=True)
    assert gn.n_rows == m and gn.n_model == nc
    p = torch.tensor(rng.standard_normal(nc), device=DEV)
    y = torch.tensor(rng.standard_normal(m), device=DEV)
    Kp, KTy = gn.apply(p), gn.apply_T(y)
    tan.status()
    assert _rel(Kp, K(p.cpu().numpy())) <= 1e-10
    assert _rel(KTy, KT(y.cpu().numpy())) <= 1e-10
    b = np.concatenate([-(wd * rng.standard_normal(wd.shape) * 1e-3).ravel(), np.zeros(m - wd.size)])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        gn.start(torch.tensor(b, device=DEV))
        gn.iterate(5, use_graph=True)
        x5, sc5 = gn.solution()
    stream.synchronize()
    xo, info = oracle_mod.lsmr(K, KT, b, 5)
    assert _rel(x5, xo) <= 1e-9
    assert abs(sc5["normr"] - info["normr"]) <= 1e-9 * info["normr"]
