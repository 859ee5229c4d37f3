"""GPU parity: libeik (through its C-ABI) against the CPU FP64 oracle on the same seeded
inputs.  Structure (SCC labels, levels, canonical order, rows) must match bit for bit
given the same frozen T; FP64 results within relative 1e-10, FP32 results (FP64 SCC
blocks) within relative 1e-5, both measured in the max norm of each output."""
import numpy as np
import pytest
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-10, torch.float32: 1e-5}
DEV = "cuda"


def rel_err(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300))


# --------------------------------------------------------------------------- cases
def _graph_case(n, A, eps, srcs):
    g = W.graph_grid(n, A)
    Ts, s = [], None
    for (a, b) in srcs:
        src = g.index(a, b, 0)
        st = W.radial_state(g, src) if eps == 0 else W.curved_state(g, src, eps)
        Ts.append(st.T)
        s = st.s if s is None else s
    # curved states derive s from T; for a multi-source tangent one slowness is shared,
    # so use the first source's (any positive s is a valid calibration input)
    return g, np.stack(Ts), s, np.array([g.index(a, b, 0) for (a, b) in srcs], dtype=np.int32)


def _config1_case(nsrc=2):
    wl = W.config1()
    g = wl.grid
    srcs = [int(wl.src[0]), g.index(45, 0)][:nsrc]
    s = 1.0 / (1.5 + 0.5 * g.xyz[:, 1])
    Ts = np.stack([W.linear_velocity_T(g.xyz, g.xyz[k], 1.5, 0.5) for k in srcs])
    return g, Ts, s, np.array(srcs, dtype=np.int32), wl.rec


def _table1_case():
    c = W.table1_case(21)
    return c.grid, c.T[None], c.s, np.array([c.src], dtype=np.int32)


CASES = {
    "cyclic-13x13x9": lambda: _graph_case((13, 13, 9), 600.0, 0.08, [(3, 3), (6, 6), (9, 3)]),
    "table3-21x21x13": lambda: _graph_case((21, 21, 13), 500.0, 0.05, [(5, 5), (10, 10)]),
    "table3-41x41x25": lambda: _graph_case((41, 41, 25), 500.0, 0.05, [(10, 10), (20, 20), (30, 10)]),
    "radialB-41x41x25": lambda: _graph_case((41, 41, 25), 600.0, 0.0, [(10, 10)]),
    "table1-21": _table1_case,
    "config1-2d": lambda: _config1_case()[:4],
}


@pytest.fixture(scope="module")
def built(oracle_mod):
    """Per case: oracle tangents and the GPU tangent of the same frozen states."""
    out = {}

    def get(name, opts=None, rec=None):
        key = (name, None if opts is None else tuple((f, getattr(opts, f)) for f, _ in opts._fields_), None if rec is None else tuple(rec))
        if key not in out:
            g, Ts, s, srcs = CASES[name]()
            _, G, _ = oracle_mod.metric(g)
            otans = [oracle_mod.build_tangent(g, G, Ts[a], s, int(srcs[a])) for a in range(len(srcs))]
            dg = eik.DeviceGrid(g)
            tan = eik.Tangent(dg, torch.tensor(Ts, device=DEV), torch.tensor(s, device=DEV), srcs, rec=rec, opts=opts)
            out[key] = (g, Ts, s, srcs, otans, tan)
        return out[key]

    return get


# --------------------------------------------------------------------------- structure
@pytest.mark.parametrize("name", list(CASES))
def test_structure_bit_exact(built, name):
    """SCC labels, levels, canonical order, level pointers and the rows of A = I - W
    (columns and FP64 weights) equal the oracle's exactly; calibration to 1 ulp-level."""
    g, Ts, s, srcs, otans, tan = built(name)
    for a, ot in enumerate(otans):
        ex = tan.export(a)
        assert np.array_equal(ex["label"], ot.label)
        assert np.array_equal(ex["level"], ot.level)
        assert np.array_equal(ex["perm"], ot.perm)
        assert np.array_equal(ex["level_ptr"], ot.level_ptr)
        assert np.array_equal(ex["row_ptr"], ot.row_ptr)
        assert np.array_equal(ex["col"], ot.col)
        assert np.array_equal(ex["w"], ot.w)
        assert np.max(np.abs(ex["cs"] - ot.cs)) <= 1e-14 * np.max(np.abs(ot.cs))
        st = ex["stats"]
        sizes = ot.scc_sizes()
        assert st["components"] == ot.ncomp and st["levels"] == ot.nlev
        assert st["nontrivial"] == int(np.sum(sizes > 1))
        assert st["largest"] == (int(sizes[sizes > 1].max()) if np.any(sizes > 1) else 0)
        assert st["edges"] == len(ot.col)


def test_table3_counts_on_gpu(built):
    """Table 3 row 41x41x25 from the GPU's own structure: 6 SCCs, 82 cyclic, largest 20."""
    _, _, _, _, _, tan = built("table3-41x41x25")
    st = tan.stats(0)
    assert (st["nontrivial"], st["cyclic_nodes"], st["largest"]) == (6, 82, 20)


# --------------------------------------------------------------------------- solves
@pytest.mark.parametrize("name", ["cyclic-13x13x9", "table3-41x41x25", "config1-2d", "table1-21"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("R", [1, 3, 8, 64])
def test_solve_primal_and_transpose(oracle_mod, built, name, dtype, R):
    """A^-1 q and A^-T r for every source (Prop. 3, Sec. 4.3) against the oracle."""
    g, Ts, s, srcs, otans, tan = built(name)
    S, N = len(srcs), g.N
    rng = np.random.default_rng(R)
    q = rng.standard_normal((S, N, R))
    qd = torch.tensor(q, device=DEV, dtype=dtype)
    x = tan.solve(qd).double().cpu().numpy()
    lam = tan.solve_T(qd).double().cpu().numpy()
    tan.status()
    qq = qd.double().cpu().numpy()   # the rounded input both sides see
    for a in range(S):
        ref = oracle_mod.solve(otans[a], qq[a])
        assert rel_err(x[a], ref) <= TOL[dtype]
        ref = oracle_mod.solve_T(otans[a], qq[a])
        assert rel_err(lam[a], ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("sched", [eik.SCHED_LEVELS, eik.SCHED_STAGED])
@pytest.mark.parametrize("R", [8, 64])
def test_levels_schedule_matches_persistent(built, dtype, sched, R):
    """The per-level schedules (graph-replayed launches, with rows in registers or staged
    in shared memory by bulk copies) and the persistent schedule run the same arithmetic
    per node; they may differ only in how the compiler fuses multiply-adds."""
    g, Ts, s, srcs, otans, tan = built("table3-41x41x25")
    tan_l = built("table3-41x41x25", opts=eik.default_opts(schedule=sched, chunk=16))[-1]
    q = torch.randn((len(srcs), g.N, R), device=DEV, dtype=dtype, generator=torch.Generator(DEV).manual_seed(5))
    tol = 1e-6 if dtype == torch.float32 else 1e-14
    for _ in range(2):                       # the second call replays the captured graph
        for f in ("solve", "solve_T"):
            a, b = getattr(tan, f)(q), getattr(tan_l, f)(q)
            assert float((a - b).abs().max() / b.abs().max()) <= tol
    tan_l.status()


@pytest.mark.parametrize("case,chunk", [("table3-41x41x25", 8), ("table3-41x41x25", 64), ("cyclic-13x13x9", 4)])
def test_item_waits_match_level_waits(built, case, chunk):
    """Persistent items that wait only for the items holding their upstream rows give
    bit-identical results to items that wait for their whole previous level (same
    kernel, same arithmetic), over repeated calls and CTA counts."""
    g, Ts, s, srcs, otans, tan = built(case, opts=eik.default_opts(chunk=chunk))
    q = torch.randn((len(srcs), g.N, 8), device=DEV, dtype=torch.float32, generator=torch.Generator(DEV).manual_seed(9))
    tan.tune(item_deps=0)
    ref = [tan.solve(q).clone(), tan.solve_T(q).clone()]
    for per_sm in (0, 1):
        tan.tune(item_deps=1, ctas_per_sm=per_sm)
        for _ in range(3):
            assert torch.equal(tan.solve(q), ref[0])
            assert torch.equal(tan.solve_T(q), ref[1])
    tan.status()


@pytest.mark.parametrize("schedule", [eik.SCHED_PERSISTENT, eik.SCHED_LEVELS, eik.SCHED_STAGED])
def test_rhs_chunking_and_tune(built, schedule):
    """Right-hand sides processed in column chunks (and options changed on a built
    tangent) give the same results as one pass."""
    g, Ts, s, srcs, otans, tan = built("cyclic-13x13x9")
    rng = np.random.default_rng(8)
    p = torch.tensor(rng.standard_normal((g.N, 24)), device=DEV, dtype=torch.float32)
    y = torch.tensor(rng.standard_normal((len(srcs), 1, 24)), device=DEV, dtype=torch.float32)
    tan_r = built("cyclic-13x13x9", rec=np.array([g.index(6, 6, 0)], dtype=np.int32))[-1]
    tan_r.tune(schedule=schedule, rhs_chunk=0)
    _, ref = tan_r.apply(p, shared_model=True)
    gref, _ = tan_r.apply_T(y, sum_sources=True)
    for chunk in (4, 8, 16):
        tan_r.tune(rhs_chunk=chunk)
        _, got = tan_r.apply(p, shared_model=True)
        gg, _ = tan_r.apply_T(y, sum_sources=True)
        assert float((got - ref).abs().max()) <= 1e-6 * float(ref.abs().max())
        assert float((gg - gref).abs().max()) <= 1e-6 * float(gref.abs().max())
    tan_r.tune(rhs_chunk=0, schedule=eik.SCHED_PERSISTENT)
    tan_r.status()


# --------------------------------------------------------------------------- J and J^T
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("model", [eik.MODEL_SLOWNESS, eik.MODEL_VELOCITY, eik.MODEL_RELATIVE])
def test_jacobian_actions(oracle_mod, dtype, model):
    """J p and J^T y with M, C, P and the source sum (Sec. 4.4) against the oracle, both
    for a model shared by all sources and for per-source right-hand sides."""
    g, Ts, s, srcs, rec = _config1_case()
    _, G, _ = oracle_mod.metric(g)
    otans = [oracle_mod.build_tangent(g, G, Ts[a], s, int(srcs[a])) for a in range(len(srcs))]
    tan = eik.Tangent(eik.DeviceGrid(g), torch.tensor(Ts, device=DEV), torch.tensor(s, device=DEV), srcs,
                      rec=rec, opts=eik.default_opts(model=model))
    S, N, R, nr = len(srcs), g.N, 4, len(rec)
    rng = np.random.default_rng(11)
    p = torch.tensor(rng.standard_normal((N, R)), device=DEV, dtype=dtype)
    pS = torch.tensor(rng.standard_normal((S, N, R)), device=DEV, dtype=dtype)
    y = torch.tensor(rng.standard_normal((S, nr, R)), device=DEV, dtype=dtype)
    dT = torch.empty((S, N, R), device=DEV, dtype=dtype)
    _, drec = tan.apply(p, shared_model=True, dT_full=dT)
    ref = oracle_mod.J(otans, s, rec, p.double().cpu().numpy(), model=model)
    assert rel_err(drec.cpu(), ref) <= TOL[dtype]
    _, drec2 = tan.apply(pS, shared_model=False)
    ref2 = oracle_mod.J(otans, s, rec, pS.double().cpu().numpy(), model=model, shared=False)
    assert rel_err(drec2.cpu(), ref2) <= TOL[dtype]
    g_sum, _ = tan.apply_T(y, sum_sources=True)
    refT = oracle_mod.JT(otans, s, rec, y.double().cpu().numpy(), model=model)
    assert rel_err(g_sum.cpu(), refT) <= TOL[dtype]
    lam = torch.empty((S, N, R), device=DEV, dtype=dtype)
    g_per, _ = tan.apply_T(y, sum_sources=False, lam_full=lam)
    refTs = oracle_mod.JT(otans, s, rec, y.double().cpu().numpy(), model=model, sum_sources=False)
    assert rel_err(g_per.cpu(), refTs) <= TOL[dtype]
    tan.status()
    # adjoint pairing on the device results themselves (Sec. 4.4)
    if dtype == torch.float64:
        l1 = float((drec * y).sum())
        l2 = float((p * g_sum).sum())
        assert abs(l1 - l2) <= 1e-13 * max(abs(l1), abs(l2))


def test_no_receivers_and_edge_sources(oracle_mod):
    """Tangent without receivers (solves only) and sources on grid corners and edges."""
    g = W.graph_grid((11, 11, 7), 300.0)
    srcs = [g.index(0, 0, 0), g.index(10, 10, 0), g.index(0, 10, 6), g.index(5, 0, 3)]
    Ts = np.stack([W.curved_state(g, k, 0.05).T for k in srcs])
    s = W.curved_state(g, srcs[0], 0.05).s
    _, G, _ = oracle_mod.metric(g)
    tan = eik.Tangent(eik.DeviceGrid(g), torch.tensor(Ts, device=DEV), torch.tensor(s, device=DEV), srcs)
    q = torch.randn((len(srcs), g.N, 2), device=DEV, dtype=torch.float64)
    x = tan.solve(q).cpu().numpy()
    for a, k in enumerate(srcs):
        ot = oracle_mod.build_tangent(g, G, Ts[a], s, k)
        assert rel_err(x[a], oracle_mod.solve(ot, q[a].cpu().numpy())) <= 1e-10
        assert np.array_equal(tan.export(a)["perm"], ot.perm)


def test_duplicate_receivers_rejected():
    g, Ts, s, srcs, rec = _config1_case(1)
    bad = np.array([rec[0], rec[0]], dtype=np.int32)
    with pytest.raises(eik.EikError) as e:
        eik.Tangent(eik.DeviceGrid(g), torch.tensor(Ts, device=DEV), torch.tensor(s, device=DEV), srcs, rec=bad)
    assert e.value.code == -1


# --------------------------------------------------------------------------- sweeping, state
@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("name", ["cyclic-13x13x9", "config1-2d"])
@pytest.mark.parametrize("dtype,R", [(torch.float64, 3), (torch.float64, 8), (torch.float32, 8), (torch.float32, 64)])
def test_sweeping_baseline_matches(oracle_mod, built, transpose, name, dtype, R):
    """Directional Gauss-Seidel sweeping (Sec. 3.6) converges to the block traversal's
    solution: to the FP64 parity tolerance in FP64 (sweep_tol 1e-13), and in FP32 to the
    FP32 tolerance of the other tests (sweep_tol 1e-7, FP32 weights and sums)."""
    g, Ts, s, srcs, otans, tan = built(name)
    q = torch.randn((len(srcs), g.N, R), device=DEV, dtype=dtype, generator=torch.Generator(DEV).manual_seed(3))
    tol = 1e-13 if dtype == torch.float64 else 1e-7
    x, cyc = tan.sweep(q, transpose=transpose, opts=eik.default_opts(sweep_tol=tol))
    x2, cyc2 = tan.sweep(q, transpose=transpose, opts=eik.default_opts(sweep_tol=tol))   # replayed cycle graph
    tan.status()
    assert cyc > 1 and cyc2 == cyc and torch.equal(x, x2)
    ref = tan.solve_T(q) if transpose else tan.solve(q)
    assert rel_err(x.cpu(), ref.cpu()) <= TOL[dtype]


def test_eik_forward_matches_oracle(oracle_mod):
    """Factored Lax-Friedrichs state (reading of Sec. 2.1-2.2): the device iterates follow
    the oracle's operation sequence, so the fixed points agree to rounding."""
    wl = W.config1()
    g = wl.grid
    dg = eik.DeviceGrid(g)
    srcs = [int(wl.src[0]), g.index(40, 0)]
    T, cyc = eik.eik_forward(dg, torch.tensor(wl.s, device=DEV), srcs)
    for a, k in enumerate(srcs):
        ref, ocyc = oracle_mod.eik_forward(g, wl.s, k)
        assert ocyc > 0
        assert rel_err(T[a].cpu(), ref) <= 1e-12
    g3 = W.graph_grid((17, 15, 9), 300.0)
    s3 = 1.0 / (2000.0 + 0.5 * g3.xyz[:, 2])
    srcs3 = [g3.index(4, 4, 0), g3.index(12, 7, 0)]
    T3, _ = eik.eik_forward(eik.DeviceGrid(g3), torch.tensor(s3, device=DEV), srcs3)
    for a, k in enumerate(srcs3):
        ref, _ = oracle_mod.eik_forward(g3, s3, k)
        assert rel_err(T3[a].cpu(), ref) <= 1e-12


def test_eik_forward_fp32_far_field(oracle_mod):
    """Precision split of the state solve: FP32 arithmetic away from the source, FP64 in
    its neighbourhood; the result stays within 1e-5 of the FP64 oracle state."""
    wl = W.config1()
    g = wl.grid
    srcs = [int(wl.src[0]), g.index(40, 0)]
    T, cyc = eik.eik_forward(eik.DeviceGrid(g), torch.tensor(wl.s, device=DEV), srcs,
                             opts=eik.default_opts(eik_fp32=1))
    for a, k in enumerate(srcs):
        ref, _ = oracle_mod.eik_forward(g, wl.s, k)
        assert rel_err(T[a].cpu(), ref) <= 1e-5
    g3, _ = W._config3d("3d", (41, 41, 21), 20.0, 8.0, 2.0, 20263)
    s3 = 1.0 / W._velocity3d(g3, 2.0)
    srcs3 = [g3.index(10, 10, 0), g3.index(30, 20, 0)]
    T3, _ = eik.eik_forward(eik.DeviceGrid(g3), torch.tensor(s3, device=DEV), srcs3,
                            opts=eik.default_opts(eik_fp32=1))
    for a, k in enumerate(srcs3):
        ref, _ = oracle_mod.eik_forward(g3, s3, k)
        assert rel_err(T3[a].cpu(), ref) <= 1e-5


def test_eik_forward_homogeneous_exact():
    """In a homogeneous medium tau = 1 is the discrete fixed point: T = s |x - x_s|."""
    g = W.table1_grid(21)
    s = np.full(g.N, 1.0 / 3000.0)
    src = g.index(10, 10, 0)
    T, cyc = eik.eik_forward(eik.DeviceGrid(g), torch.tensor(s, device=DEV), [src])
    ref = np.sqrt(((g.xyz - g.xyz[src]) ** 2).sum(1)) / 3000.0
    assert cyc == 1
    assert np.max(np.abs(T[0].cpu().numpy() - ref)) <= 1e-15 * ref.max() * 10


# --------------------------------------------------------------------------- failure paths
@pytest.mark.parametrize("chunk", [64, 8])
def test_wait_timeout_reported_and_context_survives(built, chunk):
    """A bounded device wait that can never be satisfied ends with EIK_ERR_TIMEOUT; the
    next traversal on the same context is correct again."""
    opts = eik.default_opts(wait_timeout_s=0.25, chunk=chunk)
    g, Ts, s, srcs, otans, tan = built("table3-21x21x13", opts=opts)
    q = torch.randn((len(srcs), g.N, 2), device=DEV, dtype=torch.float64)
    good = tan.solve(q).clone()
    tan.status()
    tan.debug_hold(0, 3)
    tan.solve(q)
    with pytest.raises(eik.EikError) as e:
        tan.status()
    assert e.value.code == -5
    tan.debug_hold(-1, -1)
    again = tan.solve(q)
    tan.status()
    assert torch.equal(again, good)


def test_autotuner_applies_a_setting_and_keeps_results(built, tmp_path):
    """The autotuner times the candidate settings, applies the fastest, caches it, and the
    tuned tangent computes the same J p as before."""
    from paper_2609_14982_b300.autotune import autotune
    g, Ts, s, srcs, otans, tan = built("table3-21x21x13", rec=np.array([g_i for g_i in range(0, 21 * 13, 13)], dtype=np.int32))
    p = torch.randn((g.N, 8), device=DEV, dtype=torch.float32, generator=torch.Generator(DEV).manual_seed(1))
    _, ref = tan.apply(p, shared_model=True)
    cache = str(tmp_path / "tune.json")
    rec = autotune(tan, 8, torch.float32, reps=1, cache_path=cache)
    assert rec["cached"] is False and len(rec["tried"]) >= 4
    _, got = tan.apply(p, shared_model=True)
    assert float((got - ref).abs().max()) <= 1e-6 * float(ref.abs().max())
    again = autotune(tan, 8, torch.float32, cache_path=cache)
    assert again["cached"] is True and again["setting"] == rec["setting"]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("sched,chunk", [(eik.SCHED_STAGED, 16), (eik.SCHED_PERSISTENT, 64), (eik.SCHED_PERSISTENT, 16)])
def test_staged_schedule_jacobian_against_oracle(oracle_mod, dtype, sched, chunk):
    """J p and J^T y with the staged (bulk-copy) schedule and the persistent schedule
    (shared-memory input rows at R = 64) against the oracle."""
    g, Ts, s, srcs, rec = _config1_case()
    _, G, _ = oracle_mod.metric(g)
    otans = [oracle_mod.build_tangent(g, G, Ts[a], s, int(srcs[a])) for a in range(len(srcs))]
    tan = eik.Tangent(eik.DeviceGrid(g), torch.tensor(Ts, device=DEV), torch.tensor(s, device=DEV), srcs,
                      rec=rec, opts=eik.default_opts(schedule=sched, chunk=chunk))
    rng = np.random.default_rng(12)
    p = torch.tensor(rng.standard_normal((g.N, 64)), device=DEV, dtype=dtype)
    y = torch.tensor(rng.standard_normal((len(srcs), len(rec), 64)), device=DEV, dtype=dtype)
    for _ in range(2):
        _, drec = tan.apply(p, shared_model=True)
        gs, _ = tan.apply_T(y, sum_sources=True)
    tan.status()
    assert rel_err(drec.cpu(), oracle_mod.J(otans, s, rec, p.double().cpu().numpy())) <= TOL[dtype]
    assert rel_err(gs.cpu(), oracle_mod.JT(otans, s, rec, y.double().cpu().numpy())) <= TOL[dtype]
