"""CPU FP64 oracle for the frozen full-metric Eikonal tangent transport (arxiv 2609.14982).

TEST INFRASTRUCTURE ONLY: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package.  It shares no code with the CUDA
library; both take their inputs from ``paper_2609_14982_b300.workloads``.

What it computes (paper sections in brackets):
  * metric J = dx/dxi by finite differences, G = J^-1 J^-T, mu_G      [Sec. 2.2, Eq. muG]
  * face-based upwind rows A = I - W and the calibration c^(s)        [Sec. 3.1-3.2]
  * dependency graph, SCCs (Tarjan), Kahn residual                    [Sec. 3.3-3.5, 4.1]
  * canonical condensation order and levels (longest path)            [Sec. 4.1]
  * dense partial-pivot LU of every nontrivial SCC block              [Sec. 4.3]
  * block traversals A^-1 q and A^-T r                                 [Prop. 3, Sec. 4.3]
  * the plain definition of the same solves: assembled sparse A and a
    library direct solve (numpy dense / SciPy sparse LU)              [Eq. transport-system]
  * J = P A^-1 C M and J^T = M^T C^T A^-T P^T, summed over sources     [Sec. 4.4]
  * directional sweeping (Gauss-Seidel over 2^D orderings)            [Sec. 3.6]
  * the augmented Gauss-Newton operator K, K^T (W_d, roughness R,
    relative damping S_k) and LSMR on it                               [Sec. 4.5]
  * the node <- cell averaging map of a cell-based velocity model      [Sec. 5.3]
  * multilinear sampling of off-grid receivers (P, P^T) in J, J^T      [Sec. 4.4]
  * off-grid point sources: the state from the interpolated source
    slowness, differentiated seed rows, and the direct term D_a for
    receivers inside the source cell                                  [Sec. 3.1, 3.2, 4.4]

Where the paper leaves a detail open the oracle takes one stated reading (face
averages, boundary stencils, canonical order); those readings are pinned by the
paper's printed Tables 1-3 in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_pd = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_pl = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_pi = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_pc = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc, FP64, no contraction of multiply-adds)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        I, Lg, D = C.c_int, C.c_long, C.c_double
        L.or_metric.argtypes = [I, _pi, _pd, _pd, _pd, _pd, _pd]
        L.or_grad.argtypes = [I, _pi, _pd, _pd, _pd]
        L.or_assemble.argtypes = [I, _pi, _pd, _pd, _pd, _pd, _pd, Lg, _pl, _pi, _pd, _pd, _pd, _pi]
        L.or_assemble.restype = Lg
        L.or_scc.argtypes = [Lg, _pl, _pi, _pi]
        L.or_scc.restype = Lg
        L.or_levels.argtypes = [Lg, _pl, _pi, _pi, _pi, _pi, _pl, _pl, C.POINTER(Lg)]
        L.or_levels.restype = Lg
        L.or_lu.argtypes = [I, _pd, _pi]
        L.or_lu_solve.argtypes = [I, _pd, _pi, _pd]
        L.or_lu_solve_T.argtypes = [I, _pd, _pi, _pd]
        L.or_btf_solve.argtypes = [Lg, _pl, _pi, _pd, _pi, Lg, _pl, _pl, _pd, _pi, _pl, _pd, _pd, _pd]
        L.or_btf_solve_T.argtypes = [Lg, _pl, _pi, _pd, _pi, Lg, _pl, _pl, _pd, _pi, _pl, _pd, _pd, _pd]
        L.or_sweep.argtypes = [I, _pi, I, _pl, _pi, _pd, _pd, _pd, D, Lg]
        L.or_sweep.restype = Lg
        L.or_kahn_residual.argtypes = [Lg, _pl, _pi, _pc]
        L.or_kahn_residual.restype = Lg
        L.or_eik_lf.argtypes = [I, _pi, _pd, _pd, _pd, Lg, D, D, Lg, _pd]
        L.or_eik_lf.restype = Lg
        L.or_eik_lf_point.argtypes = [I, _pi, _pd, _pd, _pd, _pd, D, D, D, Lg, _pd]
        L.or_eik_lf_point.restype = Lg
        L.or_assemble_seeds.argtypes = [I, _pi, _pd, _pd, _pd, _pd, _pd, _pl, I, _pl, _pi, _pd, _pd, _pd, _pi]
        L.or_assemble_seeds.restype = Lg
        _lib = L
    return _lib


def _n(grid):
    return np.ascontiguousarray(grid.n, dtype=np.int32), np.ascontiguousarray(grid.dxi, dtype=np.float64)


# --------------------------------------------------------------------------- metric
def metric(grid):
    """Sec. 2.2: returns (J [N,d,d], G [N,d,d], det J [N])."""
    n, dxi = _n(grid)
    N, d = grid.N, grid.ndim
    J = np.zeros((N, d, d))
    G = np.zeros((N, d, d))
    det = np.zeros(N)
    if lib().or_metric(d, n, dxi, np.ascontiguousarray(grid.xyz), J.reshape(-1), G.reshape(-1), det) != 0:
        raise ValueError("grid needs at least 3 nodes per dimension")
    return J, G, det


def mu_G(G: np.ndarray) -> float:
    """Eq. (muG): max over nodes and index pairs of |G_ab| / sqrt(G_aa G_bb)."""
    d = G.shape[1]
    best = 0.0
    for a in range(d):
        for b in range(a + 1, d):
            best = max(best, float(np.max(np.abs(G[:, a, b]) / np.sqrt(G[:, a, a] * G[:, b, b]))))
    return best


def grad(grid, f: np.ndarray) -> np.ndarray:
    n, dxi = _n(grid)
    g = np.zeros((grid.N, grid.ndim))
    lib().or_grad(grid.ndim, n, dxi, np.ascontiguousarray(f, dtype=np.float64), g.reshape(-1))
    return g


# --------------------------------------------------------------------------- tangent
@dataclass
class Tangent:
    """The frozen per-source state S_alpha = {T, A, graph, Pi, LU factors} (Sec. 4.3)."""
    N: int
    src: int
    row_ptr: np.ndarray     # gather form: upstream j of row i at col[row_ptr[i]:row_ptr[i+1]]
    col: np.ndarray
    c: np.ndarray           # coupling magnitudes c_ij
    w: np.ndarray           # normalized weights w_ij
    cs: np.ndarray          # calibration c^(s)_i (0 on the seed row)
    row_type: np.ndarray    # 0 interior, 1 seed, 2 identity (no upstream face)
    label: np.ndarray = None      # SCC label = smallest node of the component
    level: np.ndarray = None      # level of the node's component
    perm: np.ndarray = None       # position -> node (canonical order)
    comp_ptr: np.ndarray = None
    level_ptr: np.ndarray = None
    ncomp: int = 0
    nlev: int = 0
    lu_off: np.ndarray = None
    lu: np.ndarray = None
    piv: np.ndarray = None
    piv_off: np.ndarray = None
    cptr: np.ndarray = None       # column (transpose) form
    crow: np.ndarray = None
    cw: np.ndarray = None

    def A(self):
        """Assembled sparse A = I - W (Eq. transport-system)."""
        import scipy.sparse as sp
        rows = np.repeat(np.arange(self.N), np.diff(self.row_ptr))
        W = sp.csr_matrix((self.w, (rows, self.col)), shape=(self.N, self.N))
        return (sp.identity(self.N, format="csr") - W).tocsr()

    def edges(self):
        """(j, i) pairs of the dependency graph: edge j -> i iff w_ij > 0 (Sec. 3.3)."""
        rows = np.repeat(np.arange(self.N), np.diff(self.row_ptr))
        return self.col.astype(np.int64), rows

    # -- structure statistics (Sec. 5.2, Eq. graph-fractions)
    def scc_sizes(self) -> np.ndarray:
        _, counts = np.unique(self.label, return_counts=True)
        return counts

    def kahn_unresolved(self) -> int:
        rem = np.zeros(self.N, dtype=np.int8)
        return int(lib().or_kahn_residual(self.N, self.row_ptr, self.col, rem))

    def kahn_removed(self) -> np.ndarray:
        rem = np.zeros(self.N, dtype=np.int8)
        lib().or_kahn_residual(self.N, self.row_ptr, self.col, rem)
        return rem.astype(bool)


def assemble(grid, G, T, s, src, seeds=None) -> Tangent:
    """Sec. 3.1-3.2: upwind rows and calibration for one source state T.  The seed rows
    (identities) are the source node, or the given seed nodes of a point source."""
    n, dxi = _n(grid)
    N = grid.N
    gT = grad(grid, T)
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    cap = 2 * grid.ndim * N
    col = np.zeros(cap, dtype=np.int32)
    cw = np.zeros(cap)
    w = np.zeros(cap)
    cs = np.zeros(N)
    rt = np.zeros(N, dtype=np.int32)
    if seeds is None:
        nnz = lib().or_assemble(grid.ndim, n, dxi, np.ascontiguousarray(G.reshape(-1)), gT.reshape(-1),
                                np.ascontiguousarray(T, dtype=np.float64), np.ascontiguousarray(s, dtype=np.float64),
                                int(src), row_ptr, col, cw, w, cs, rt)
    else:
        sd = np.ascontiguousarray(seeds, dtype=np.int64)
        nnz = lib().or_assemble_seeds(grid.ndim, n, dxi, np.ascontiguousarray(G.reshape(-1)), gT.reshape(-1),
                                      np.ascontiguousarray(T, dtype=np.float64),
                                      np.ascontiguousarray(s, dtype=np.float64), sd, len(sd), row_ptr, col, cw, w,
                                      cs, rt)
    if nnz < 0:
        raise ValueError("assembly failed")
    return Tangent(N, int(src), row_ptr, col[:nnz].copy(), cw[:nnz].copy(), w[:nnz].copy(), cs, rt)


def condense(t: Tangent) -> Tangent:
    """Sec. 4.1: SCC labels, canonical levels/order, and LU factors of the nontrivial blocks."""
    L = lib()
    N = t.N
    label = np.zeros(N, dtype=np.int32)
    L.or_scc(N, t.row_ptr, t.col, label)
    level = np.zeros(N, dtype=np.int32)
    perm = np.zeros(N, dtype=np.int32)
    comp_ptr = np.zeros(N + 1, dtype=np.int64)
    level_ptr = np.zeros(N + 1, dtype=np.int64)
    nc = C.c_long(0)
    nlev = L.or_levels(N, t.row_ptr, t.col, label, level, perm, comp_ptr, level_ptr, C.byref(nc))
    if nlev < 0:
        raise RuntimeError("condensation is not acyclic" if nlev == -1 else "grid too large for the oracle key")
    ncomp = nc.value
    t.label, t.level, t.perm = label, level, perm
    t.comp_ptr = comp_ptr[:ncomp + 1].copy()
    t.level_ptr = level_ptr[:nlev + 1].copy()
    t.ncomp, t.nlev = ncomp, int(nlev)
    # LU of nontrivial blocks (nodes ascending inside a block)
    sizes = np.diff(t.comp_ptr)
    lu_off = np.full(ncomp, -1, dtype=np.int64)
    piv_off = np.full(ncomp, -1, dtype=np.int64)
    blocks = np.nonzero(sizes > 1)[0]
    tot = int(np.sum(sizes[blocks].astype(np.int64) ** 2))
    lu = np.zeros(max(tot, 1))
    piv = np.zeros(max(int(np.sum(sizes[blocks])), 1), dtype=np.int32)
    o = po = 0
    for c in blocks:
        k = int(sizes[c])
        nodes = perm[t.comp_ptr[c]:t.comp_ptr[c + 1]]
        Ac = block_matrix(t, nodes)
        a = np.ascontiguousarray(Ac.reshape(-1))
        p = np.zeros(k, dtype=np.int32)
        if L.or_lu(k, a, p) != 0:
            raise np.linalg.LinAlgError(f"singular SCC block of size {k}")
        lu[o:o + k * k] = a
        piv[po:po + k] = p
        lu_off[c] = o
        piv_off[c] = po
        o += k * k
        po += k
    t.lu_off, t.lu, t.piv, t.piv_off = lu_off, lu, piv, piv_off
    # transpose (column) form
    rows = np.repeat(np.arange(N, dtype=np.int32), np.diff(t.row_ptr))
    order = np.argsort(t.col, kind="stable")
    t.crow = rows[order].astype(np.int32)
    t.cw = t.w[order].copy()
    cnt = np.bincount(t.col, minlength=N)
    t.cptr = np.zeros(N + 1, dtype=np.int64)
    t.cptr[1:] = np.cumsum(cnt)
    return t


def block_matrix(t: Tangent, nodes: np.ndarray) -> np.ndarray:
    """A_C = I - W_CC for a component (nodes ascending), Sec. 4.2."""
    k = len(nodes)
    where = {int(v): a for a, v in enumerate(nodes)}
    Ac = np.eye(k)
    for a, i in enumerate(nodes):
        for e in range(t.row_ptr[i], t.row_ptr[i + 1]):
            b = where.get(int(t.col[e]))
            if b is not None:
                Ac[a, b] -= t.w[e]
    return Ac


def build_tangent(grid, G, T, s, src) -> Tangent:
    return condense(assemble(grid, G, T, s, src))


# --------------------------------------------------------------------------- point sources
@dataclass
class PointSource:
    """A source between grid nodes.  The paper supplies its source rows from a
    differentiated source treatment (Sec. 3.1, 3.2) without printing it; reading:
      * the source sits at fractional logical coordinates f; its cell has corner base
        b_d = min(floor(f_d), n_d - 2) and local coordinates t = f - b; corner o (in the
        order of itertools.product((0, 1), repeat=ndim)) has the multilinear weight
        phi_o = prod_d (t_d if o_d else 1 - t_d), the product taken axis by axis;
      * position x_src = sum_o phi_o x_o and slowness s_src = sum_o phi_o s_o, each summed
        in corner order;
      * the state is the factored solve with T0 = s_src |x - x_src|, every corner kept at
        T = T0 (their distances r_o = |x_o - x_src|);
      * the corners are the seed rows of A (identities), and differentiating T_o = s_src r_o
        gives their right-hand side q_o = r_o sum_k phi_k ds_k."""
    f: np.ndarray
    nodes: np.ndarray
    phi: np.ndarray
    x: np.ndarray
    s_src: float
    r: np.ndarray


def _cell(grid, f):
    import itertools
    nd = grid.ndim
    n = [int(v) for v in grid.n[:nd]]
    f = [float(v) for v in f]
    base = [min(int(np.floor(f[d])), n[d] - 2) for d in range(nd)]
    t = [f[d] - base[d] for d in range(nd)]
    nodes, phi = [], []
    for o in itertools.product((0, 1), repeat=nd):
        idx = [base[d] + o[d] for d in range(nd)]
        node = 0
        for d in range(nd):
            node = node * n[d] + idx[d]
        w = 1.0
        for d in range(nd):
            w = w * (t[d] if o[d] else 1.0 - t[d])
        nodes.append(node)
        phi.append(w)
    return np.array(nodes, dtype=np.int64), np.array(phi), tuple(base)


def point_source(grid, s, f) -> PointSource:
    nd = grid.ndim
    for d in range(nd):
        if not (0.0 <= float(f[d]) <= grid.n[d] - 1):
            raise ValueError("source coordinate out of the grid")
    nodes, phi, _ = _cell(grid, f)
    x = np.zeros(nd)
    s_src = 0.0
    for k in range(len(nodes)):
        for c in range(nd):
            x[c] = x[c] + phi[k] * grid.xyz[nodes[k], c]
        s_src = s_src + phi[k] * float(s[nodes[k]])
    r = np.zeros(len(nodes))
    for k in range(len(nodes)):
        acc = 0.0
        for c in range(nd):
            d = grid.xyz[nodes[k], c] - x[c]
            acc = acc + d * d
        r[k] = np.sqrt(acc)
    return PointSource(np.asarray(f, dtype=np.float64), nodes, phi, x, s_src, r)


def eik_forward_point(grid, s, f, radius=1.0, tol=1e-12, max_cycles=2000):
    """The factored state of a point source (PointSource's reading).  Nodes within
    max(radius x largest spacing, largest corner distance) of x_src keep tau = 1, so
    every seed corner holds T = s_src r exactly.  Returns (T [N], cycles, PointSource)."""
    ps = point_source(grid, s, f)
    n, dxi = _n(grid)
    rad = max(float(radius) * max(grid.dxi), float(ps.r.max()))
    T = np.zeros(grid.N)
    cyc = lib().or_eik_lf_point(grid.ndim, n, dxi, np.ascontiguousarray(grid.xyz),
                                np.ascontiguousarray(s, dtype=np.float64), np.ascontiguousarray(ps.x),
                                float(ps.s_src), rad, float(tol), int(max_cycles), T)
    return T, int(cyc), ps


def build_tangent_point(grid, G, T, s, ps: PointSource) -> Tangent:
    """The tangent of a point source: its cell corners are the seed rows."""
    t = condense(assemble(grid, G, T, s, -1, seeds=ps.nodes))
    t.ps = ps
    return t


def source_rhs(t: Tangent, ds: np.ndarray) -> np.ndarray:
    """q = C ds (Sec. 3.2): q_i = c_i ds_i off the seeds; on a point source's seed rows
    q_o = r_o sum_k phi_k ds_k (differentiated source treatment).  ds [N, R]."""
    q = t.cs[:, None] * ds
    ps = getattr(t, "ps", None)
    if ps is not None:
        sigma = ps.phi @ ds[ps.nodes]
        q[ps.nodes] += ps.r[:, None] * sigma[None, :]
    return q


def source_rhs_T(t: Tangent, lam: np.ndarray) -> np.ndarray:
    """C^T lam, the transpose of source_rhs.  lam [N, R]."""
    out = t.cs[:, None] * lam
    ps = getattr(t, "ps", None)
    if ps is not None:
        tau = ps.r @ lam[ps.nodes]
        out[ps.nodes] += ps.phi[:, None] * tau[None, :]
    return out


def direct_term(grid, ps: PointSource, f_rec: np.ndarray):
    """D_a of Eq. (source-jacobian) for off-grid receivers (reading): a receiver in the
    source's cell is predicted by the source treatment itself, T_r = s_src |x_r - x_src|
    (x_r the multilinear image of its fractional coordinates), so its row of D is
    |x_r - x_src| phi (on the corners) and its row of P is zero; every other receiver has
    a zero row of D.  Returns (D as CSR [n_rec, N], boolean mask of the direct receivers)."""
    import scipy.sparse as sp
    f_rec = np.asarray(f_rec, dtype=np.float64)
    _, _, sbase = _cell(grid, ps.f)
    rows, cols, vals = [], [], []
    direct = np.zeros(len(f_rec), dtype=bool)
    for j, fr in enumerate(f_rec):
        nodes, phi, base = _cell(grid, fr)
        if base != sbase:
            continue
        direct[j] = True
        xr = np.zeros(grid.ndim)
        for k in range(len(nodes)):
            for c in range(grid.ndim):
                xr[c] = xr[c] + phi[k] * grid.xyz[nodes[k], c]
        rho = float(np.sqrt(np.sum((xr - ps.x) ** 2)))
        for k in range(len(ps.nodes)):
            rows.append(j)
            cols.append(int(ps.nodes[k]))
            vals.append(rho * ps.phi[k])
    D = sp.csr_matrix((vals, (rows, cols)), shape=(len(f_rec), grid.N))
    return D, direct


# --------------------------------------------------------------------------- solves
def solve(t: Tangent, q: np.ndarray) -> np.ndarray:
    """x = A^-1 q by block traversal (Prop. 3).  q: [N] or [N, R]."""
    q = np.asarray(q, dtype=np.float64)
    if q.ndim == 2:
        return np.stack([solve(t, q[:, r]) for r in range(q.shape[1])], axis=1)
    x = np.zeros(t.N)
    work = np.zeros(max(int(np.max(np.diff(t.comp_ptr))), 1))
    lib().or_btf_solve(t.N, t.row_ptr, t.col, t.w, t.perm, t.ncomp, t.comp_ptr, t.lu_off, t.lu,
                       t.piv, t.piv_off, np.ascontiguousarray(q), x, work)
    return x


def solve_T(t: Tangent, r: np.ndarray) -> np.ndarray:
    """lam = A^-T r by reverse block traversal with U^T, L^T, P^T (Sec. 4.3)."""
    r = np.asarray(r, dtype=np.float64)
    if r.ndim == 2:
        return np.stack([solve_T(t, r[:, k]) for k in range(r.shape[1])], axis=1)
    lam = np.zeros(t.N)
    work = np.zeros(max(int(np.max(np.diff(t.comp_ptr))), 1))
    lib().or_btf_solve_T(t.N, t.cptr, t.crow, t.cw, t.perm, t.ncomp, t.comp_ptr, t.lu_off, t.lu,
                         t.piv, t.piv_off, np.ascontiguousarray(r), lam, work)
    return lam


def direct_solve(t: Tangent, q: np.ndarray, transpose: bool = False) -> np.ndarray:
    """The plain definition: assemble A and call a library direct solver."""
    A = t.A()
    if transpose:
        A = A.T.tocsc()
    if t.N <= 3000:
        return np.linalg.solve(A.toarray(), q)
    import scipy.sparse.linalg as spla
    return spla.splu(A.tocsc()).solve(np.asarray(q, dtype=np.float64))


def sweep(grid, t: Tangent, b: np.ndarray, transpose=False, tol=1e-12, max_cycles=100000):
    """Sec. 3.6: directional Gauss-Seidel sweeping; returns (x, cycles)."""
    n, _ = _n(grid)
    x = np.zeros(t.N)
    if transpose:
        cyc = lib().or_sweep(grid.ndim, n, 1, t.cptr, t.crow, t.cw, np.ascontiguousarray(b, dtype=np.float64),
                             x, tol, max_cycles)
    else:
        cyc = lib().or_sweep(grid.ndim, n, 0, t.row_ptr, t.col, t.w, np.ascontiguousarray(b, dtype=np.float64),
                             x, tol, max_cycles)
    return x, int(cyc)


# --------------------------------------------------------------------------- state
def eik_forward(grid, s, src, radius=1.0, tol=1e-12, max_cycles=2000):
    """Sec. 2.1-2.2 (reading): factored full-metric Lax-Friedrichs sweeping for one source.
    radius is in units of the largest logical spacing.  Returns (T [N], cycles)."""
    n, dxi = _n(grid)
    T = np.zeros(grid.N)
    cyc = lib().or_eik_lf(grid.ndim, n, dxi, np.ascontiguousarray(grid.xyz), np.ascontiguousarray(s, dtype=np.float64),
                          int(src), float(radius) * max(grid.dxi), float(tol), int(max_cycles), T)
    return T, int(cyc)


# --------------------------------------------------------------------------- maps and J
MODEL_SLOWNESS, MODEL_VELOCITY, MODEL_RELATIVE = 0, 1, 2


def model_factor(s: np.ndarray, model: int) -> np.ndarray:
    """M (Sec. 2.3): ds = p (slowness), ds = -s^2 dv (velocity), ds = -s m (relative)."""
    if model == MODEL_SLOWNESS:
        return np.ones_like(s)
    if model == MODEL_VELOCITY:
        return -s * s
    return -s


def J(tans, s, rec, p, model=MODEL_SLOWNESS, shared=True, solver=solve):
    """Eq. (source-jacobian) with D = 0: J_a p = P A_a^-1 C_a M p for every source.
    p: [N, R] (shared model) or [S, N, R]; rec: [n_rec] node indices.
    Returns d_rec [S, n_rec, R]."""
    m = model_factor(s, model)
    out = []
    for a, t in enumerate(tans):
        pa = p if shared else p[a]
        pa = pa if pa.ndim == 2 else pa[:, None]
        ds = m[:, None] * pa
        dT = solver(t, source_rhs(t, ds))
        out.append(dT[np.asarray(rec)])
    return np.stack(out)


def JT(tans, s, rec, y, model=MODEL_SLOWNESS, sum_sources=True, solver=solve_T):
    """Eq. (source-transpose) with D = 0: J_a^T y_a = M^T C^T A_a^-T P^T y_a, summed over
    sources when sum_sources.  y: [S, n_rec, R].  Returns [N, R] or [S, N, R]."""
    m = model_factor(s, model)
    outs = []
    for a, t in enumerate(tans):
        r = np.zeros((t.N, y.shape[2]))
        np.add.at(r, np.asarray(rec), y[a])
        lam = solver(t, r)
        outs.append(m[:, None] * source_rhs_T(t, lam))
    outs = np.stack(outs)
    return outs.sum(axis=0) if sum_sources else outs


# --------------------------------------------------------------------------- LSQR
def lsqr(apply_J, apply_JT, b: np.ndarray, iters: int):
    """LSQR (Paige and Saunders, 1982), plain numpy, x0 = 0, no damping: the Krylov
    least-squares loop that Sec. 4.5 runs on the paired actions.  Returns (x, phibar)."""
    beta = np.linalg.norm(b)
    u = b / beta
    v = apply_JT(u)
    alpha = np.linalg.norm(v)
    v = v / alpha
    w = v.copy()
    x = np.zeros_like(v)
    phibar, rhobar = beta, alpha
    for _ in range(iters):
        u = apply_J(v) - alpha * u
        beta = np.linalg.norm(u)
        u = u / beta
        v = apply_JT(u) - beta * v
        alpha = np.linalg.norm(v)
        v = v / alpha
        rho = np.hypot(rhobar, beta)
        c, s = rhobar / rho, beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        x = x + (phi / rho) * w
        w = v - (theta / rho) * w
    return x, phibar


# --------------------------------------------------------------------------- Sec. 4.5
def roughness(grid):
    """R, the model-increment roughness operator of Eq. (gn-subproblem).  The paper does
    not define it; reading: first differences along every logical axis, unit weight,
    (R p)_row = p[i + e_d] - p[i] for every node pair adjacent along axis d.  Rows are
    ordered axis by axis, and within an axis by the linear index of the lower node.
    Returns a scipy.sparse CSR matrix [n_rough, N]."""
    import scipy.sparse as sp
    n = tuple(int(x) for x in grid.n[:grid.ndim])
    N = int(np.prod(n))
    idx = np.arange(N).reshape(n)
    rows, cols, vals = [], [], []
    r0 = 0
    for d in range(len(n)):
        lo = np.take(idx, np.arange(n[d] - 1), axis=d).ravel()
        hi = np.take(idx, np.arange(1, n[d]), axis=d).ravel()
        order = np.argsort(lo, kind="stable")
        lo, hi = lo[order], hi[order]
        m = len(lo)
        r = r0 + np.arange(m)
        rows += [r, r]
        cols += [hi, lo]
        vals += [np.ones(m), -np.ones(m)]
        r0 += m
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(r0, N))


def gn_operator(grid, tans, s, rec, wd, vk, lam, gamma, model=MODEL_VELOCITY, cells=False):
    """The augmented Gauss-Newton operator of Eq. (augmented-actions):
        K p   = [W_d J p ; lam R p ; lam S p],        S = gamma diag(1 / v_k)  (Eq. relative-damping)
        K^T y = J^T W_d y_d + lam R^T y_R + lam S^T y_S.
    wd: [S, n_rec] diagonal of W_d; vk: the current model.  With cells=True the model
    lives on the cells (cell_average): J acts through A (J A p, A^T J^T y), R takes first
    differences on the cell grid and vk is [n_cells].  p is the model vector; y is
    [S*n_rec + n_rough + n_model].  Returns (apply_K, apply_KT, n_rows)."""
    if cells:
        A = cell_average(grid)
        cgrid = type("CellGrid", (), {"ndim": grid.ndim, "n": tuple(m - 1 for m in grid.n[:grid.ndim])})()
        Rm = roughness(cgrid)
    else:
        A = None
        Rm = roughness(grid)
    S_, nr = len(tans), len(rec)
    nd, nR, N = S_ * nr, Rm.shape[0], len(vk)
    sdiag = gamma / np.asarray(vk, dtype=np.float64)

    def apply_K(p):
        pn = A @ p if cells else p
        d = J(tans, s, rec, pn[:, None], model=model)[:, :, 0] * wd
        return np.concatenate([d.ravel(), lam * (Rm @ p), lam * sdiag * p])

    def apply_KT(y):
        yd = (y[:nd].reshape(S_, nr) * wd)[:, :, None]
        g = JT(tans, s, rec, yd, model=model)[:, 0]
        if cells:
            g = A.T @ g
        return g + lam * (Rm.T @ y[nd:nd + nR]) + lam * sdiag * y[nd + nR:]

    return apply_K, apply_KT, nd + nR + N


def lsmr(apply_A, apply_AT, b: np.ndarray, iters: int):
    """LSMR (Fong and Saunders, 2011), plain numpy, x0 = 0, no damping: the Krylov solver
    that Sec. 4.5 applies to the augmented system.  Golub-Kahan bidiagonalization, the
    first QR (rotations P_k) of B_k, the second QR (rotations Pbar_k) of [R_k^T; theta e_k^T],
    and x updated through the h, hbar recurrences.  The residual norm |b - A x_k| is
    carried by a third rotation sequence (Ptilde) applied to R_bar^T and to the rotated
    right-hand side; |A^T r_k| = |zetabar_{k+1}|.
    Returns (x, info) with info = {normr, normar, norma, normx, iters}."""
    beta = np.linalg.norm(b)
    u = b / beta
    v = apply_AT(u)
    alpha = np.linalg.norm(v)
    v = v / alpha
    x = np.zeros_like(v)
    h = v.copy()
    hbar = np.zeros_like(v)
    alphabar, zetabar = alpha, alpha * beta
    rho, rhobar, cbar, sbar, zeta = 1.0, 1.0, 1.0, 0.0, 0.0
    # residual-norm recurrences
    betadd, betad, rhodot, thetatilde, tautilde_prev, done2 = beta, 0.0, 1.0, 0.0, 0.0, 0.0
    norma2 = alpha * alpha
    normr = beta
    for _ in range(iters):
        u = apply_A(v) - alpha * u
        beta = np.linalg.norm(u)
        u = u / beta
        v = apply_AT(u) - beta * v
        alpha = np.linalg.norm(v)
        v = v / alpha
        norma2 += beta * beta + alpha * alpha
        # P_k: eliminate beta_{k+1} from B_k
        rho_prev = rho
        rho = np.hypot(alphabar, beta)
        c, s = alphabar / rho, beta / rho
        theta = s * alpha
        alphabar = c * alpha
        # Pbar_k: eliminate theta_{k+1} from [R_k^T; theta e_k^T]
        rhobar_prev, zeta_prev = rhobar, zeta
        thetabar = sbar * rho
        rhobar = np.hypot(cbar * rho, theta)
        cbar, sbar = cbar * rho / rhobar, theta / rhobar
        zeta = cbar * zetabar
        zetabar = -sbar * zetabar
        # h, hbar, x
        hbar = h - (thetabar * rho / (rho_prev * rhobar_prev)) * hbar
        x = x + (zeta / (rho * rhobar)) * hbar
        h = v - (theta / rho) * h
        # |r_k|: P_k on the right-hand side, then Ptilde_{k-1} on Rbar^T and on it
        betahat = c * betadd
        betadd = -s * betadd
        rhotilde = np.hypot(rhodot, thetabar)
        ctilde, stilde = rhodot / rhotilde, thetabar / rhotilde
        thetatilde_prev = thetatilde
        thetatilde = stilde * rhobar
        rhodot = ctilde * rhobar
        betatilde = ctilde * betad + stilde * betahat
        betad = -stilde * betad + ctilde * betahat
        tautilde = (zeta_prev - thetatilde_prev * tautilde_prev) / rhotilde
        taudot = (zeta - thetatilde * tautilde) / rhodot
        done2 += (betatilde - tautilde) ** 2
        tautilde_prev = tautilde
        normr = np.sqrt(done2 + (betad - taudot) ** 2 + betadd ** 2)
    info = {"normr": float(normr), "normar": float(abs(zetabar)), "norma": float(np.sqrt(norma2)),
            "normx": float(np.linalg.norm(x)), "iters": iters}
    return x, info


# --------------------------------------------------------------------------- cell model
def cell_average(grid):
    """Node <- cell map of a cell-based velocity model (the paper's inversion cells,
    Sec. 5.3: one cell per grid hexahedron).  Reading (the paper gives no formula): a
    node's velocity perturbation is the mean of its adjacent cells' perturbations,
    dv_node[j] = (1 / n_adj(j)) sum over the cells c with j as a corner of dv_cell[c].
    Cells are indexed like nodes on the grid of extents n_d - 1.  Returns a scipy.sparse
    CSR matrix [N, n_cells]; the model map of J is then M = -s^2 (velocity) times it."""
    import itertools

    import scipy.sparse as sp
    n = tuple(int(x) for x in grid.n[:grid.ndim])
    m = tuple(x - 1 for x in n)
    nc = int(np.prod(m))
    cidx = np.arange(nc).reshape(m)
    rows, cols = [], []
    for off in itertools.product((0, 1), repeat=len(n)):
        sl = tuple(slice(o, o + mm) for o, mm in zip(off, m))
        nodes = np.arange(int(np.prod(n))).reshape(n)[sl]
        rows.append(nodes.ravel())
        cols.append(cidx.ravel())
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    nadj = np.bincount(rows, minlength=int(np.prod(n))).astype(np.float64)
    return sp.csr_matrix((1.0 / nadj[rows], (rows, cols)), shape=(int(np.prod(n)), nc))


# --------------------------------------------------------------------------- off-grid receivers
def receiver_interp(grid, f: np.ndarray):
    """Multilinear receiver sampling P (Sec. 4.4's P_a for receivers off the grid nodes;
    the paper gives no formula, reading: multilinear interpolation in logical index space).
    f: [n_rec, ndim] fractional logical indices, 0 <= f_d <= n_d - 1.  Corner base
    b_d = min(floor(f_d), n_d - 2), t_d = f_d - b_d, weight of corner o in {0,1}^ndim
    = prod_d (t_d if o_d else 1 - t_d).  Returns a scipy.sparse CSR matrix [n_rec, N]."""
    import itertools

    import scipy.sparse as sp
    f = np.asarray(f, dtype=np.float64)
    n = np.array(grid.n[:grid.ndim])
    base = np.minimum(np.floor(f).astype(np.int64), n - 2)
    t = f - base
    strides = np.array([int(np.prod(n[d + 1:])) for d in range(grid.ndim)])
    rows, cols, vals = [], [], []
    for o in itertools.product((0, 1), repeat=grid.ndim):
        o = np.array(o)
        w = np.prod(np.where(o == 1, t, 1.0 - t), axis=1)
        rows.append(np.arange(len(f)))
        cols.append(((base + o) * strides).sum(axis=1))
        vals.append(w)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(len(f), int(np.prod(n))))


def J_interp(tans, s, Ps, p, model=MODEL_SLOWNESS, Ds=None):
    """Eq. (source-jacobian): J_a p = (P_a A_a^-1 C_a + D_a) M p with a sparse P_a per
    source (D_a = 0 unless given); p [N, R] shared.  Returns [S, n_rec, R]."""
    m = model_factor(s, model)
    out = []
    for a, (t, P) in enumerate(zip(tans, Ps)):
        ds = m[:, None] * p
        d = P @ solve(t, source_rhs(t, ds))
        if Ds is not None and Ds[a] is not None:
            d = d + Ds[a] @ ds
        out.append(d)
    return np.stack(out)


def JT_interp(tans, s, Ps, y, model=MODEL_SLOWNESS, Ds=None):
    """Eq. (source-transpose) summed over sources: sum_a M^T (C_a^T A_a^-T P_a^T y_a +
    D_a^T y_a); y [S, n_rec, R].  Returns [N, R]."""
    m = model_factor(s, model)
    g = 0.0
    for a, (t, P) in enumerate(zip(tans, Ps)):
        h = source_rhs_T(t, solve_T(t, P.T @ y[a]))
        if Ds is not None and Ds[a] is not None:
            h = h + Ds[a].T @ y[a]
        g = g + m[:, None] * h
    return g
