"""Thin Python binding of libeik (include/eik.h): argument marshalling only.

Every call passes device pointers of torch CUDA tensors and torch's current CUDA
stream to the C-ABI; all arithmetic runs in the library's CUDA kernels.  There is no
CPU or PyTorch fallback: without the built library (libeik.so next to this file) or
without a CUDA device every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
# EIK_LIB selects another build of the library, e.g. the checked build (build.py --checked)
LIB_PATH = os.environ.get("EIK_LIB") or os.path.join(HERE, "libeik.so")

EIK_F64, EIK_F32 = 0, 1
MODEL_SLOWNESS, MODEL_VELOCITY, MODEL_RELATIVE = 0, 1, 2
SCHED_PERSISTENT, SCHED_LEVELS, SCHED_STAGED, SCHED_CLUSTER, SCHED_SYNC = 0, 1, 2, 3, 4
STATUS = {0: "OK", -1: "INVALID", -2: "OOM", -3: "SINGULAR_BLOCK", -4: "NOT_CONVERGED", -5: "TIMEOUT",
          -6: "CUDA", -7: "CYCLE"}

EXPORTED = ["eik_opts_default", "eik_last_error", "eik_version", "eik_forward", "tangent_build", "tangent_apply",
            "tangent_apply_T", "tangent_solve", "tangent_solve_T", "tangent_sample", "tangent_stats", "tangent_dims",
            "tangent_export", "tangent_status", "tangent_free", "sweep_apply", "tangent_debug_hold", "tangent_tune",
            "lsqr_create", "lsqr_start", "lsqr_iterate", "lsqr_solution", "lsqr_free",
            "eik_forward_noalloc", "eik_forward_noalloc_capacity",
            "gn_create", "gn_dims", "gn_apply", "gn_apply_T", "gn_lsmr_start", "gn_lsmr_iterate",
            "gn_lsmr_solution", "gn_free", "model_cells_to_nodes", "model_nodes_to_cells",
            "tangent_set_receivers", "tangent_apply_interp", "tangent_apply_interp_T", "gn_create_cells", "gn_rhs",
            "tangent_apply_batch", "tangent_apply_T_batch", "eik_forward_points", "tangent_build_points",
            "eik_forward_warm", "tangent_debug_poke_edge"]


class EikError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libeik {STATUS.get(code, code)}: {msg}")
        self.code = code


class Grid_(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("dxi", C.c_double * 3), ("xyz", C.c_void_p)]


class Opts(C.Structure):
    _fields_ = [("model", C.c_int), ("lu_pivot_tol", C.c_double), ("schedule", C.c_int), ("threads", C.c_int),
                ("chunk", C.c_int), ("ctas_per_sm", C.c_int), ("wait_timeout_s", C.c_double),
                ("eik_tol", C.c_double), ("eik_max_cycles", C.c_int), ("eik_src_radius", C.c_double),
                ("sweep_tol", C.c_double), ("sweep_max_cycles", C.c_int), ("rhs_chunk", C.c_int),
                ("eik_fp32", C.c_int), ("eik_fp64_radius", C.c_double), ("item_deps", C.c_int),
                ("cluster_size", C.c_int), ("cluster_threads", C.c_int), ("pass_units", C.c_int),
                ("block_lu_min", C.c_int), ("split_dirs", C.c_int), ("item_slots", C.c_int)]


class Stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("nodes", "edges", "components", "nontrivial", "cyclic_nodes", "largest",
                                         "levels", "max_level_width", "identity_rows", "lu_doubles")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


_lib = None


def lib():
    """Load libeik.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_2609_14982_b300.build`")
        L = C.CDLL(LIB_PATH)
        P, I, D = C.c_void_p, C.c_int, C.c_double
        L.eik_opts_default.argtypes = [C.POINTER(Opts)]
        L.eik_last_error.restype = C.c_char_p
        L.eik_version.restype = C.c_char_p
        L.eik_forward.argtypes = [C.POINTER(Grid_), P, I, P, P, C.POINTER(Opts), C.POINTER(I), P]
        L.eik_forward_noalloc.argtypes = [C.POINTER(Grid_), P, I, P, P, C.POINTER(Opts), C.POINTER(I), P]
        L.eik_forward_noalloc_capacity.restype = C.c_size_t
        L.tangent_build.argtypes = [C.POINTER(Grid_), P, P, I, P, P, I, C.POINTER(Opts), C.POINTER(P), P]
        L.tangent_build_points.argtypes = [C.POINTER(Grid_), P, P, I, P, P, I, C.POINTER(Opts), C.POINTER(P), P]
        L.eik_forward_points.argtypes = [C.POINTER(Grid_), P, I, P, P, C.POINTER(Opts), C.POINTER(I), P]
        L.eik_forward_warm.argtypes = [C.POINTER(Grid_), P, I, P, P, P, C.POINTER(Opts), C.POINTER(I), P]
        L.tangent_apply.argtypes = [P, P, I, I, P, P, I, P]
        L.tangent_apply_T.argtypes = [P, P, I, I, P, P, I, P]
        L.tangent_solve.argtypes = [P, P, I, P, I, P]
        L.tangent_solve_T.argtypes = [P, P, I, P, I, P]
        L.tangent_sample.argtypes = [P, P, P, P]
        L.tangent_stats.argtypes = [P, I, C.POINTER(Stats)]
        L.tangent_dims.argtypes = [P, C.POINTER(I), C.POINTER(C.c_int64), C.POINTER(I)]
        L.tangent_export.argtypes = [P, I, P, P, P, P, P, P, P, P]
        L.tangent_status.argtypes = [P, P]
        L.tangent_free.argtypes = [P]
        L.tangent_free.restype = None
        L.tangent_debug_hold.argtypes = [P, I, I]
        L.tangent_debug_poke_edge.argtypes = [P, I, C.c_longlong, I]
        L.tangent_tune.argtypes = [P, C.POINTER(Opts)]
        L.lsqr_create.argtypes = [P, I, C.POINTER(P)]
        L.lsqr_start.argtypes = [P, P, P]
        L.lsqr_iterate.argtypes = [P, I, I, P]
        L.lsqr_solution.argtypes = [P, P, P, P]
        L.lsqr_free.argtypes = [P]
        L.lsqr_free.restype = None
        L.gn_create.argtypes = [P, P, P, D, D, I, C.POINTER(P)]
        L.gn_create_cells.argtypes = [P, P, P, D, D, I, C.POINTER(P)]
        L.gn_dims.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.gn_apply.argtypes = [P, P, P, P]
        L.gn_apply_T.argtypes = [P, P, P, P]
        L.gn_lsmr_start.argtypes = [P, P, P]
        L.gn_rhs.argtypes = [P, P, P, P]
        L.tangent_apply_batch.argtypes = [P, I, P, P, P, I, P]
        L.tangent_apply_T_batch.argtypes = [P, I, P, P, P, I, P]
        L.gn_lsmr_iterate.argtypes = [P, I, I, P]
        L.gn_lsmr_solution.argtypes = [P, P, P, P]
        L.gn_free.argtypes = [P]
        L.gn_free.restype = None
        L.model_cells_to_nodes.argtypes = [C.POINTER(Grid_), P, I, P, I, P]
        L.tangent_set_receivers.argtypes = [P, I, P]
        L.tangent_apply_interp.argtypes = [P, P, I, I, P, I, P]
        L.tangent_apply_interp_T.argtypes = [P, P, I, P, I, P]
        L.model_nodes_to_cells.argtypes = [C.POINTER(Grid_), P, I, P, I, P]
        L.sweep_apply.argtypes = [P, I, P, I, P, I, C.POINTER(Opts), C.POINTER(I), P]
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise EikError(rc, lib().eik_last_error().decode())


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().eik_opts_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t: torch.Tensor, dtype=None, name="tensor") -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return t.data_ptr()


def _dt(dtype) -> int:
    if dtype == torch.float64:
        return EIK_F64
    if dtype == torch.float32:
        return EIK_F32
    raise TypeError("dtype must be float32 or float64")


class DeviceGrid:
    """A workload grid on the device (xyz float64 [N, ndim])."""

    def __init__(self, grid, device="cuda"):
        self.host = grid
        self.ndim = grid.ndim
        self.n = tuple(grid.n)
        self.N = grid.N
        self.xyz = torch.as_tensor(grid.xyz, dtype=torch.float64, device=device).contiguous()
        self.c = Grid_()
        self.c.ndim = grid.ndim
        for d in range(3):
            self.c.n[d] = grid.n[d] if d < grid.ndim else 1
            self.c.dxi[d] = grid.dxi[d] if d < grid.ndim else 1.0
        self.c.xyz = self.xyz.data_ptr()


def n_cells(dgrid: DeviceGrid) -> int:
    out = 1
    for m in dgrid.n[:dgrid.ndim]:
        out *= m - 1
    return out


def cells_to_nodes(dgrid: DeviceGrid, p_cell: torch.Tensor) -> torch.Tensor:
    """Node perturbations [N, R] from cell perturbations [n_cells, R] (mean over adjacent cells)."""
    pc = p_cell if p_cell.dim() == 2 else p_cell[:, None]
    out = torch.empty((dgrid.N, pc.shape[1]), dtype=pc.dtype, device=pc.device)
    _check(lib().model_cells_to_nodes(C.byref(dgrid.c), _dev(pc), int(pc.shape[1]), _dev(out, pc.dtype, "out"),
                                      _dt(pc.dtype), _stream()))
    return out if p_cell.dim() == 2 else out[:, 0]


def nodes_to_cells(dgrid: DeviceGrid, g_node: torch.Tensor) -> torch.Tensor:
    """Transpose of cells_to_nodes: [N, R] -> [n_cells, R]."""
    gn = g_node if g_node.dim() == 2 else g_node[:, None]
    out = torch.empty((n_cells(dgrid), gn.shape[1]), dtype=gn.dtype, device=gn.device)
    _check(lib().model_nodes_to_cells(C.byref(dgrid.c), _dev(gn), int(gn.shape[1]), _dev(out, gn.dtype, "out"),
                                      _dt(gn.dtype), _stream()))
    return out if g_node.dim() == 2 else out[:, 0]


def _check_state_args(dgrid: DeviceGrid, s: torch.Tensor, S: int, out: torch.Tensor | None):
    """Shapes and devices of a state solve, checked before any pointer reaches the library:
    s has N entries, out is [S, N], and s, out and the grid live on the current device."""
    if int(s.numel()) != dgrid.N:
        raise ValueError(f"s has {int(s.numel())} entries, the grid has {dgrid.N} nodes")
    if out is not None and tuple(out.shape) != (S, dgrid.N):
        raise ValueError(f"out must be [{S}, {dgrid.N}], got {list(out.shape)}")
    if s.is_cuda:
        cur = torch.cuda.current_device()
        for name, t in (("s", s), ("out", out), ("grid", dgrid.xyz)):
            if t is not None and t.is_cuda and t.device.index != cur:
                raise ValueError(f"{name} is on {t.device}, the current device is cuda:{cur}")


def eik_forward(dgrid: DeviceGrid, s: torch.Tensor, src, opts: Opts | None = None, out: torch.Tensor | None = None,
                T_init: torch.Tensor | None = None):
    """First-arrival traveltimes [S, N] (float64) for the given source nodes; with T_init
    [S, N] the sweeps start from that field (eik_forward_warm)."""
    src = torch.as_tensor(src, dtype=torch.int32).contiguous().cpu()
    S = int(src.numel())
    _check_state_args(dgrid, s, S, out)
    if out is None:
        out = torch.empty((S, dgrid.N), dtype=torch.float64, device=s.device)
    cyc = C.c_int(0)
    if T_init is not None:
        _check_state_args(dgrid, s, S, T_init)
        _check(lib().eik_forward_warm(C.byref(dgrid.c), _dev(s, torch.float64, "s"), S, C.c_void_p(src.data_ptr()),
                                      _dev(T_init, torch.float64, "T_init"), _dev(out, torch.float64, "T"),
                                      C.byref(opts) if opts else None, C.byref(cyc), _stream()))
        return out, cyc.value
    _check(lib().eik_forward(C.byref(dgrid.c), _dev(s, torch.float64, "s"), S, C.c_void_p(src.data_ptr()),
                             _dev(out, torch.float64, "T"), C.byref(opts) if opts else None, C.byref(cyc), _stream()))
    return out, cyc.value


def _points(dgrid: DeviceGrid, src_f) -> torch.Tensor:
    f = torch.as_tensor(src_f, dtype=torch.float64).cpu()
    if f.dim() == 1:
        f = f.unsqueeze(0)
    if f.dim() != 2 or f.shape[1] != dgrid.c.ndim:
        raise ValueError(f"point sources must be [S, {dgrid.c.ndim}] fractional logical coordinates")
    return f.contiguous()


def eik_forward_points(dgrid: DeviceGrid, s: torch.Tensor, src_f, opts: Opts | None = None,
                       out: torch.Tensor | None = None):
    """First-arrival traveltimes [S, N] (float64) for point sources at fractional logical
    coordinates src_f [S, ndim]."""
    f = _points(dgrid, src_f)
    S = int(f.shape[0])
    _check_state_args(dgrid, s, S, out)
    if out is None:
        out = torch.empty((S, dgrid.N), dtype=torch.float64, device=s.device)
    cyc = C.c_int(0)
    _check(lib().eik_forward_points(C.byref(dgrid.c), _dev(s, torch.float64, "s"), S, C.c_void_p(f.data_ptr()),
                                    _dev(out, torch.float64, "T"), C.byref(opts) if opts else None, C.byref(cyc),
                                    _stream()))
    return out, cyc.value


def eik_forward_noalloc(dgrid: DeviceGrid, s: torch.Tensor, src, out: torch.Tensor, opts: Opts | None = None):
    """Same result as eik_forward, without any device allocation inside the library: the
    caller provides T [S, N] (float64) and the scratch is the library's fixed array."""
    src = torch.as_tensor(src, dtype=torch.int32).contiguous().cpu()
    _check_state_args(dgrid, s, int(src.numel()), out)
    cyc = C.c_int(0)
    _check(lib().eik_forward_noalloc(C.byref(dgrid.c), _dev(s, torch.float64, "s"), int(src.numel()),
                                     C.c_void_p(src.data_ptr()), _dev(out, torch.float64, "T"),
                                     C.byref(opts) if opts else None, C.byref(cyc), _stream()))
    return out, cyc.value


class Tangent:
    """The frozen per-source states S_a of all sources (owned by libeik)."""

    def __init__(self, dgrid: DeviceGrid, T: torch.Tensor, s: torch.Tensor, src, rec=None, opts: Opts | None = None,
                 points: bool = False):
        """src: source nodes [S], or with points=True fractional logical coordinates [S, ndim]
        of point sources (tangent_build_points)."""
        if points:
            src = _points(dgrid, src)
            self.S = int(src.shape[0])
        else:
            src = torch.as_tensor(src, dtype=torch.int32).contiguous().cpu()
            self.S = int(src.numel())
        if rec is None:
            rec = torch.zeros((self.S, 0), dtype=torch.int32)
        rec = torch.as_tensor(rec, dtype=torch.int32).cpu()
        if rec.dim() == 1:
            rec = rec.unsqueeze(0).expand(self.S, -1)
        rec = rec.contiguous()
        self.n_rec = int(rec.shape[1])
        self.N = dgrid.N
        self.dgrid = dgrid
        self.opts = opts if opts is not None else default_opts()
        h = C.c_void_p()
        build = lib().tangent_build_points if points else lib().tangent_build
        _check(build(C.byref(dgrid.c), _dev(T, torch.float64, "T"), _dev(s, torch.float64, "s"),
                     self.S, C.c_void_p(src.data_ptr()),
                     C.c_void_p(rec.data_ptr()) if self.n_rec else None, self.n_rec,
                     C.byref(self.opts), C.byref(h), _stream()))
        self.h = h

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "h", None) and self.h.value:
            lib().tangent_free(self.h)
            self.h = C.c_void_p()

    # ---- Jacobian actions
    def apply(self, p: torch.Tensor, shared_model: bool, dT_full=None, d_rec=None):
        """J p: p [N, R] (shared) or [S, N, R]; returns (dT_full, d_rec)."""
        R = p.shape[-1]
        if d_rec is None and self.n_rec:
            d_rec = torch.empty((self.S, self.n_rec, R), dtype=p.dtype, device=p.device)
        _check(lib().tangent_apply(self.h, _dev(p, name="p"), int(shared_model), R,
                                   _dev(dT_full, p.dtype, "dT_full") if dT_full is not None else None,
                                   _dev(d_rec, p.dtype, "d_rec") if d_rec is not None else None, _dt(p.dtype),
                                   _stream()))
        return dT_full, d_rec

    def apply_T(self, y: torch.Tensor, sum_sources: bool = True, g=None, lam_full=None, accumulate: bool = False):
        """J^T y: y [S, n_rec, R]; returns (g, lam_full).  With accumulate (and
        sum_sources) the source sum is added to the given g instead of replacing it."""
        R = y.shape[-1]
        if accumulate and (g is None or not sum_sources):
            raise ValueError("accumulate needs sum_sources and an existing g")
        if g is None:
            shape = (self.N, R) if sum_sources else (self.S, self.N, R)
            g = torch.empty(shape, dtype=y.dtype, device=y.device)
        mode = 2 if accumulate else int(bool(sum_sources))
        _check(lib().tangent_apply_T(self.h, _dev(y, name="y"), R, mode, _dev(g, y.dtype, "g"),
                                     _dev(lam_full, y.dtype, "lam_full") if lam_full is not None else None,
                                     _dt(y.dtype), _stream()))
        return g, lam_full

    def set_receivers(self, f):
        """Off-grid receivers: f [S, n_rec, ndim] fractional logical indices (host array)."""
        import numpy as np
        f = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
        assert f.ndim == 3 and f.shape[0] == self.S
        self.n_ip = int(f.shape[1])
        _check(lib().tangent_set_receivers(self.h, self.n_ip, C.c_void_p(f.ctypes.data)))

    def apply_interp(self, p: torch.Tensor, shared_model: bool = True):
        """J p sampled at the off-grid receivers: returns [S, n_rec, R]."""
        R = p.shape[-1]
        out = torch.empty((self.S, self.n_ip, R), dtype=p.dtype, device=p.device)
        _check(lib().tangent_apply_interp(self.h, _dev(p, name="p"), int(shared_model), R, _dev(out, p.dtype, "d_rec"),
                                          _dt(p.dtype), _stream()))
        return out

    def apply_interp_T(self, y: torch.Tensor):
        """J^T y for data at the off-grid receivers y [S, n_rec, R]: returns [N, R]."""
        R = y.shape[-1]
        g = torch.empty((self.N, R), dtype=y.dtype, device=y.device)
        _check(lib().tangent_apply_interp_T(self.h, _dev(y, name="y"), R, _dev(g, y.dtype, "g"), _dt(y.dtype),
                                            _stream()))
        return g

    def solve(self, q: torch.Tensor, out=None):
        """A^-1 q for every source: q [S, N, R]."""
        out = torch.empty_like(q) if out is None else out
        _check(lib().tangent_solve(self.h, _dev(q, name="q"), q.shape[-1], _dev(out, q.dtype, "x"), _dt(q.dtype),
                                   _stream()))
        return out

    def solve_T(self, r: torch.Tensor, out=None):
        out = torch.empty_like(r) if out is None else out
        _check(lib().tangent_solve_T(self.h, _dev(r, name="r"), r.shape[-1], _dev(out, r.dtype, "x"), _dt(r.dtype),
                                     _stream()))
        return out

    def sample(self, field: torch.Tensor, out=None):
        """P_a: values of a per-source FP64 field [S, N] at each source's receivers."""
        out = torch.empty((self.S, self.n_rec), dtype=torch.float64, device=field.device) if out is None else out
        _check(lib().tangent_sample(self.h, _dev(field, torch.float64, "field"), _dev(out, torch.float64, "out"),
                                    _stream()))
        return out

    def sweep(self, b: torch.Tensor, transpose=False, opts: Opts | None = None, out=None):
        """Directional Gauss-Seidel sweeping of the same operator; returns (x, cycles)."""
        out = torch.empty_like(b) if out is None else out
        cyc = C.c_int(0)
        _check(lib().sweep_apply(self.h, int(transpose), _dev(b, name="b"), b.shape[-1], _dev(out, b.dtype, "x"),
                                 _dt(b.dtype), C.byref(opts) if opts else None, C.byref(cyc), _stream()))
        return out, cyc.value

    def tune(self, **kw):
        """Change run-time options (schedule, ctas_per_sm, rhs_chunk, wait_timeout_s, item_deps,
        cluster_size, cluster_threads, pass_units, block_lu_min, split_dirs, item_slots)."""
        for k, v in kw.items():
            if k not in ("schedule", "ctas_per_sm", "rhs_chunk", "wait_timeout_s", "item_deps", "cluster_size",
                         "cluster_threads", "pass_units", "block_lu_min", "split_dirs", "item_slots"):
                raise KeyError(k)
            setattr(self.opts, k, v)
        _check(lib().tangent_tune(self.h, C.byref(self.opts)))

    def debug_poke_edge(self, source: int, edge: int, value: int):
        """Test hook of the checked build: overwrite one upstream edge's position."""
        _check(lib().tangent_debug_poke_edge(self.h, source, edge, value))

    def debug_hold(self, source: int, step: int):
        """Test hook: make the persistent traversal's wait before (source, step) run out."""
        _check(lib().tangent_debug_hold(self.h, source, step))

    # ---- structure
    def status(self):
        _check(lib().tangent_status(self.h, _stream()))

    def stats(self, a: int) -> dict:
        st = Stats()
        _check(lib().tangent_stats(self.h, a, C.byref(st)))
        return st.as_dict()

    def export(self, a: int) -> dict:
        import numpy as np
        st = self.stats(a)
        N = self.N
        label = np.zeros(N, dtype=np.int32)
        level = np.zeros(N, dtype=np.int32)
        perm = np.zeros(N, dtype=np.int32)
        level_ptr = np.zeros(st["levels"] + 1, dtype=np.int64)
        row_ptr = np.zeros(N + 1, dtype=np.int64)
        col = np.zeros(max(st["edges"], 1), dtype=np.int32)
        w = np.zeros(max(st["edges"], 1), dtype=np.float64)
        cs = np.zeros(N, dtype=np.float64)
        ptrs = [x.ctypes.data_as(C.c_void_p) for x in (label, level, perm, level_ptr, row_ptr, col, w, cs)]
        _check(lib().tangent_export(self.h, a, *ptrs))
        return dict(label=label, level=level, perm=perm, level_ptr=level_ptr, row_ptr=row_ptr,
                    col=col[:st["edges"]], w=w[:st["edges"]], cs=cs, stats=st)


def _batch(fn, tans, xs, outs):
    n = len(tans)
    if not 1 <= n <= 4 or len(xs) != n or len(outs) != n:
        raise ValueError("a batch holds 1..4 tangents with one input and one output each")
    dtype = xs[0].dtype
    th = (C.c_void_p * n)(*[t.h.value for t in tans])
    xp = (C.c_void_p * n)(*[_dev(x, dtype, "input") for x in xs])
    op = (C.c_void_p * n)(*[_dev(o, dtype, "output") for o in outs])
    rr = (C.c_int * n)(*[int(x.shape[-1]) for x in xs])
    _check(fn(th, n, xp, rr, op, _dt(dtype), _stream()))
    return outs


def apply_batch(tans, ps):
    """J p of several tangents (e.g. one per grid) in one launch: ps[k] [N_k, R_k] shared
    model blocks; returns the d_rec [S_k, n_rec_k, R_k] of each."""
    outs = [torch.empty((t.S, t.n_rec, p.shape[-1]), dtype=p.dtype, device=p.device) for t, p in zip(tans, ps)]
    return _batch(lib().tangent_apply_batch, tans, ps, outs)


def apply_T_batch(tans, ys):
    """J^T y summed over sources for several tangents in one launch: ys[k]
    [S_k, n_rec_k, R_k]; returns the g [N_k, R_k] of each."""
    outs = [torch.empty((t.N, y.shape[-1]), dtype=y.dtype, device=y.device) for t, y in zip(tans, ys)]
    return _batch(lib().tangent_apply_T_batch, tans, ys, outs)


class LSQR:
    """Device LSQR on J of a tangent (one right-hand side, slowness-type model)."""

    def __init__(self, tan: Tangent, dtype=torch.float64):
        self.tan = tan
        self.dtype = dtype
        h = C.c_void_p()
        _check(lib().lsqr_create(tan.h, _dt(dtype), C.byref(h)))
        self.h = h

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "h", None) and self.h.value:
            lib().lsqr_free(self.h)
            self.h = C.c_void_p()

    def start(self, b: torch.Tensor):
        _check(lib().lsqr_start(self.h, _dev(b, self.dtype, "b"), _stream()))

    def iterate(self, iters: int, use_graph: bool = True):
        _check(lib().lsqr_iterate(self.h, iters, int(use_graph), _stream()))

    def solution(self):
        x = torch.empty(self.tan.N, dtype=self.dtype, device="cuda")
        sc = (C.c_double * 9)()
        _check(lib().lsqr_solution(self.h, _dev(x, self.dtype, "x"), sc, _stream()))
        names = ("alpha", "beta", "rhobar", "phibar", "phi", "rho", "theta", "c", "s")
        return x, dict(zip(names, list(sc)))


class GN:
    """The augmented Gauss-Newton operator K = [W_d J; lam R; lam S_k] of a tangent and
    device LSMR on it (one model vector).  wd: [S, n_rec] FP64 data weights (diagonal of
    W_d); vk: [N] FP64 current model (S_k = gamma diag(1 / vk))."""

    def __init__(self, tan: Tangent, wd: torch.Tensor, vk: torch.Tensor, lam: float, gamma: float,
                 dtype=torch.float64, cells: bool = False):
        self.tan = tan
        self.dtype = dtype
        self.n_model = int(vk.numel())    # nodes, or cells when cells=True
        h = C.c_void_p()
        create = lib().gn_create_cells if cells else lib().gn_create
        _check(create(tan.h, _dev(wd, torch.float64, "wd"), _dev(vk, torch.float64, "vk"), float(lam),
                      float(gamma), _dt(dtype), C.byref(h)))
        self.h = h
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().gn_dims(self.h, C.byref(a), C.byref(b), C.byref(c)))
        self.n_rows, self.n_data, self.n_rough = a.value, b.value, c.value

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "h", None) and self.h.value:
            lib().gn_free(self.h)
            self.h = C.c_void_p()

    def apply(self, p: torch.Tensor) -> torch.Tensor:
        out = torch.empty(self.n_rows, dtype=self.dtype, device="cuda")
        _check(lib().gn_apply(self.h, _dev(p, self.dtype, "p"), _dev(out, self.dtype, "out"), _stream()))
        return out

    def apply_T(self, y: torch.Tensor) -> torch.Tensor:
        out = torch.empty(self.n_model, dtype=self.dtype, device="cuda")
        _check(lib().gn_apply_T(self.h, _dev(y, self.dtype, "y"), _dev(out, self.dtype, "out"), _stream()))
        return out

    def rhs(self, r: torch.Tensor) -> torch.Tensor:
        """b = [-W_d r; 0; 0] of Eq. (augmented-ls) for a residual r [S, n_rec] (FP64),
        formed on the device with the solver's own copy of W_d."""
        b = torch.empty(self.n_rows, dtype=self.dtype, device="cuda")
        _check(lib().gn_rhs(self.h, _dev(r.contiguous(), torch.float64, "r"), _dev(b, self.dtype, "b"), _stream()))
        return b

    def start(self, b: torch.Tensor):
        _check(lib().gn_lsmr_start(self.h, _dev(b, self.dtype, "b"), _stream()))

    def iterate(self, iters: int, use_graph: bool = True):
        _check(lib().gn_lsmr_iterate(self.h, iters, int(use_graph), _stream()))

    def solution(self):
        x = torch.empty(self.n_model, dtype=self.dtype, device="cuda")
        sc = (C.c_double * 6)()
        _check(lib().gn_lsmr_solution(self.h, _dev(x, self.dtype, "x"), sc, _stream()))
        names = ("normr", "normar", "norma", "normx", "normb", "iters")
        return x, dict(zip(names, list(sc)))

    def lsmr(self, b: torch.Tensor, atol: float = 1e-4, max_iters: int = 200, check_every: int = 5,
             use_graph: bool = True):
        """LSMR until |K^T r| <= atol |K| |r| (checked every `check_every` iterations) or
        max_iters; returns (x, scalars).  With use_graph the iterations are replayed from
        a CUDA graph, which needs a current stream other than the legacy default one."""
        self.start(b)
        done = 0
        while done < max_iters:
            k = min(check_every, max_iters - done)
            self.iterate(k, use_graph)
            done += k
            x, sc = self.solution()
            if sc["normar"] <= atol * sc["norma"] * sc["normr"]:
                break
        return x, sc
