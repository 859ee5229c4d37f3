"""GPU: the two ways a strongly connected block A_C is solved in the block-triangular
traversal (Sec. 4.3): multiplication by the explicit inverse formed from the block's
partial-pivot LU factors, and FP64 forward/back substitution with those factors (the
tier for large blocks, selected by block_lu_min).  On the steep-hill stress grid, whose
cyclic components are the largest of the workloads, both tiers are compared with the
oracle (which solves each block with its own LU), with each other, and across the
persistent and cluster schedules."""
import numpy as np
import pytest
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def steep(oracle_mod):
    wl = W.config5_grid(0)
    g = wl.grid
    src = wl.src[[0, 13, 31]]
    dg = eik.DeviceGrid(g)
    s = torch.tensor(wl.s, device=DEV)
    T, _ = eik.eik_forward(dg, s, src)
    Tn = T.cpu().numpy()
    _, G, _ = oracle_mod.metric(g)
    otans = [oracle_mod.build_tangent(g, G, Tn[a], wl.s, int(src[a])) for a in range(len(src))]
    return wl, g, dg, s, T, src, otans


def _rel(a, b):
    a = a.double().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _run(steep, dtype, lu_min, schedule=eik.SCHED_PERSISTENT, R=8):
    wl, g, dg, s, T, src, _ = steep
    tan = eik.Tangent(dg, T, s, src, rec=wl.rec, opts=eik.default_opts(block_lu_min=lu_min, schedule=schedule))
    rng = np.random.default_rng(77)
    p = torch.tensor(rng.standard_normal((g.N, R)), device=DEV, dtype=dtype)
    y = torch.tensor(rng.standard_normal((len(src), len(wl.rec), R)), device=DEV, dtype=dtype)
    dT = torch.empty((len(src), g.N, R), device=DEV, dtype=dtype)
    _, drec = tan.apply(p, shared_model=True, dT_full=dT)
    ga, _ = tan.apply_T(y, sum_sources=False)
    tan.status()
    st = [tan.stats(a) for a in range(len(src))]
    tan.free()
    return p, y, dT, drec, ga, st


def test_stress_grid_has_multi_node_blocks(steep):
    """The case exercises the substitution tier: every source has cyclic blocks, and the
    largest spans more than one warp's worth of rows."""
    *_, st = _run(steep, torch.float64, 0, R=1)
    assert all(x["nontrivial"] > 0 for x in st)
    assert max(x["largest"] for x in st) > 32


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_lu_substitution_matches_oracle_and_inverse(oracle_mod, steep, dtype):
    """block_lu_min = 2 solves every cyclic block by substitution: J p at the receivers,
    the full dT field and each source's J_a^T y_a agree with the oracle, and with the
    explicit-inverse tier (block_lu_min = 0) to within the rounding of the two block
    solves."""
    wl, g, dg, s, T, src, otans = steep
    p, y, dT_lu, rec_lu, ga_lu, _ = _run(steep, dtype, 2)
    _, _, dT_inv, rec_inv, ga_inv, _ = _run(steep, dtype, 0)
    tol = 1e-10 if dtype == torch.float64 else 1e-5
    pn, yn = p.double().cpu().numpy(), y.double().cpu().numpy()
    assert _rel(rec_lu, oracle_mod.J(otans, wl.s, wl.rec, pn)) <= tol
    for a in range(len(src)):
        ref = oracle_mod.JT([otans[a]], wl.s, wl.rec, yn[a:a + 1])
        assert _rel(ga_lu[a], ref) <= tol, a
    close = 1e-11 if dtype == torch.float64 else 1e-5
    assert _rel(dT_lu, dT_inv.double().cpu().numpy()) <= close
    assert _rel(ga_lu, ga_inv.double().cpu().numpy()) <= close


def test_lu_tier_same_bits_in_both_schedules(steep):
    """The cluster schedule runs the same block solve: with the substitution tier on, its
    J p and J^T y equal the persistent schedule's bit for bit."""
    out = {}
    for sched in (eik.SCHED_PERSISTENT, eik.SCHED_CLUSTER):
        _, _, dT, rec, ga, _ = _run(steep, torch.float32, 2, schedule=sched)
        out[sched] = (dT, rec, ga)
    for u, v in zip(out[eik.SCHED_PERSISTENT], out[eik.SCHED_CLUSTER]):
        assert torch.equal(u, v)


def test_lu_threshold_selects_by_block_size(steep):
    """A threshold above the largest block leaves every block on the inverse tier: the
    result equals block_lu_min = 0 bit for bit."""
    *_, st = _run(steep, torch.float64, 0, R=1)
    big = max(x["largest"] for x in st) + 1
    a = _run(steep, torch.float64, 0)
    b = _run(steep, torch.float64, big)
    for u, v in zip(a[2:5], b[2:5]):
        assert torch.equal(u, v)
