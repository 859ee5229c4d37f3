"""Seeded synthetic inputs: deformed grids, media, sources, receivers, right-hand sides.

This module holds input recipes only. It computes no part of the method (no metric,
no upwind coefficients, no graph, no solve); both the CUDA path and the CPU oracle
take their inputs from here.

Conventions
-----------
* Logical dimensions: 3-D (xi, eta, zeta), 2-D (xi, zeta). zeta is always the last
  dimension, zeta = 0 is the top (free) surface, zeta = H the flat base.
* Node linear index: 3-D (i, j, k) -> (i*n1 + j)*n2 + k, 2-D (i, k) -> i*n1 + k.
* Physical coordinates: x (and y) equal the horizontal logical coordinates; z is
  depth, positive downwards, z = zeta + (1 - zeta/H) * zsurf(x, y) (the map of
  Sec. 5.1, Eq. (test-map), and Sec. 5.2, Eq. (graph-map)), where zsurf is the
  depth of the top surface.  For the benchmark workloads the topography is given as
  an elevation e (positive up), so zsurf = -e and "depth" in a velocity law is z
  measured from the datum z = 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Grid:
    ndim: int
    n: tuple            # nodes per logical dimension
    dxi: tuple          # logical spacing per dimension
    xyz: np.ndarray     # [N, ndim] float64 physical coordinates (x[, y], z)
    lo: tuple = ()      # logical origin per dimension
    H: float = 0.0      # logical depth of the zeta axis

    @property
    def N(self) -> int:
        return int(np.prod(self.n))

    def index(self, *ijk) -> int:
        if self.ndim == 3:
            i, j, k = ijk
            return (i * self.n[1] + j) * self.n[2] + k
        i, k = ijk
        return i * self.n[1] + k

    def logical(self) -> list:
        return [self.lo[d] + self.dxi[d] * np.arange(self.n[d]) for d in range(self.ndim)]


def mapped_grid(n, lo_h, hi_h, H, zsurf) -> Grid:
    """Boundary-conforming grid x = xi, z = zeta + (1 - zeta/H) zsurf(xi).

    n: node counts (last = zeta); lo_h/hi_h: horizontal extents; zsurf: callable on
    horizontal coordinate arrays returning the depth of the top surface."""
    ndim = len(n)
    dxi = [(hi_h[d] - lo_h[d]) / (n[d] - 1) for d in range(ndim - 1)] + [H / (n[-1] - 1)]
    lo = list(lo_h) + [0.0]
    axes = [lo[d] + dxi[d] * np.arange(n[d]) for d in range(ndim)]
    mesh = np.meshgrid(*axes, indexing="ij")
    horiz = mesh[:-1]
    zeta = mesh[-1]
    zs = zsurf(*horiz)
    z = zeta + (1.0 - zeta / H) * zs
    xyz = np.stack([m.reshape(-1) for m in horiz] + [z.reshape(-1)], axis=1)
    return Grid(ndim, tuple(int(v) for v in n), tuple(float(v) for v in dxi),
                np.ascontiguousarray(xyz, dtype=np.float64), tuple(lo), float(H))


# ---------------------------------------------------------------------------
# Sec. 5.1: manufactured point-source tangent on the sinusoidal map (Table 1)
# ---------------------------------------------------------------------------
T1_L, T1_H, T1_A, T1_V0 = 4000.0, 2000.0, 200.0, 3000.0
T1_C = (0.02, 0.04, -0.03, 0.02)


def table1_grid(nx: int) -> Grid:
    """Grid of Sec. 5.1 (Eq. test-map, test-topo): xi, eta in [-L/2, L/2], zeta in [0, H],
    nx x nx x (nx+1)/2 nodes (21x21x11 ... 161x161x81), A = 200 m."""
    L, H, A = T1_L, T1_H, T1_A

    def zs(x, y):
        return A * np.sin(2 * np.pi * x / L) * np.sin(2 * np.pi * y / L)

    return mapped_grid((nx, nx, (nx + 1) // 2), (-L / 2, -L / 2), (L / 2, L / 2), H, zs)


@dataclass
class Table1Case:
    grid: Grid
    s: np.ndarray        # [N] slowness (homogeneous)
    T: np.ndarray        # [N] analytic first arrival s0 * r (Eq. test-T)
    src: int             # centre logical node
    ds: np.ndarray       # [N] linear slowness perturbation (Eq. test-ds)
    dT_exact: np.ndarray  # [N] Eq. (test-dT)
    mask: np.ndarray     # [N] bool, retained error set C_h


def table1_case(nx: int) -> Table1Case:
    g = table1_grid(nx)
    s0 = 1.0 / T1_V0
    c = g.n[0] // 2
    src = g.index(c, c, g.n[2] // 2)
    xs = g.xyz[src]
    d = g.xyz - xs
    r = np.sqrt((d * d).sum(axis=1))
    T = s0 * r
    c0, cx, cy, cz = T1_C
    ds = s0 * (c0 + cx * d[:, 0] / T1_L + cy * d[:, 1] / T1_L + cz * d[:, 2] / T1_H)
    ds_src = s0 * c0
    dT_ex = 0.5 * r * (ds_src + ds)
    h = max(g.dxi)
    idx = np.stack(np.meshgrid(*[np.arange(m) for m in g.n], indexing="ij"), -1).reshape(-1, 3)
    interior = np.all((idx > 0) & (idx < np.array(g.n) - 1), axis=1)
    mask = interior & (r > 3.0 * h)
    mask[src] = False
    return Table1Case(g, np.full(g.N, s0), T, src, ds, dT_ex, mask)


# ---------------------------------------------------------------------------
# Sec. 5.2: controlled dependency-structure cases (Tables 2 and 3)
# ---------------------------------------------------------------------------
G_L, G_H, G_V0 = 4000.0, 2000.0, 3000.0


def graph_grid(n, A: float) -> Grid:
    """Grid of Eq. (graph-map): 4 km x 4 km x 2 km, surface A sin(2 pi x/Lx) sin(2 pi y/Ly)."""
    L, H = G_L, G_H

    def zs(x, y):
        return A * np.sin(2 * np.pi * x / L) * np.sin(2 * np.pi * y / L)

    return mapped_grid(tuple(n), (-L / 2, -L / 2), (L / 2, L / 2), H, zs)


def closed_cycle_case(seed: int = 21):
    """A frozen state whose dependency graph has a closed cyclic component: a seeded random
    traveltime field (uniform noise plus a 0.3 depth trend) on a 9 x 9 grid sheared by
    z_top = c x / 2 (c ~ U(0.5, 2) from the seed), unit slowness, source at node 0.  With
    seed 21 one nontrivial SCC of 4 nodes has all its upwind faces inside itself, so its
    rows of W sum to 1 and A_C = I - W_CC is singular, the case the local-invertibility
    theorem of Sec. 4.2 excludes.  Returns (grid, T, s, src)."""
    rng = np.random.default_rng(seed)
    shear = rng.uniform(0.5, 2.0)
    g = mapped_grid((9, 9), (0.0,), (8.0,), 8.0, lambda x: shear * x * 0.5)
    T = rng.uniform(0, 1, g.N) + 0.3 * g.xyz[:, 1]
    return g, T, np.ones(g.N), 0


def quarter_source(g: Grid) -> int:
    """Surface node at logical (x, y) = (-L/4, -L/4)."""
    return g.index((g.n[0] - 1) // 4, (g.n[1] - 1) // 4, 0)


def centre_source(g: Grid) -> int:
    return g.index((g.n[0] - 1) // 2, (g.n[1] - 1) // 2, 0)


@dataclass
class StateCase:
    grid: Grid
    s: np.ndarray
    T: np.ndarray
    src: int


def radial_state(g: Grid, src: int) -> StateCase:
    """Eq. (radial-state): T = |x - x_s| / v0, homogeneous slowness."""
    d = g.xyz - g.xyz[src]
    r = np.sqrt((d * d).sum(axis=1))
    return StateCase(g, np.full(g.N, 1.0 / G_V0), r / G_V0, src)


def curved_state(g: Grid, src: int, eps: float) -> StateCase:
    """Eq. (curved-state): T = r/v0 + eps sin(4 pi X/Lx) sin(4 pi Y/Ly) sin(pi z/H) - C_s,
    X = x + Lx/2, Y = y + Ly/2, with s = |grad_x T| (analytic)."""
    L, H, v0 = G_L, G_H, G_V0
    x, y, z = g.xyz[:, 0], g.xyz[:, 1], g.xyz[:, 2]
    X, Y = x + L / 2, y + L / 2
    a, b, c = 4 * np.pi / L, 4 * np.pi / L, np.pi / H
    pert = eps * np.sin(a * X) * np.sin(b * Y) * np.sin(c * z)
    d = g.xyz - g.xyz[src]
    r = np.sqrt((d * d).sum(axis=1))
    T = r / v0 + pert - pert[src]
    rs = np.where(r > 0, r, 1.0)
    grad = d / (rs[:, None] * v0)
    grad[:, 0] += eps * a * np.cos(a * X) * np.sin(b * Y) * np.sin(c * z)
    grad[:, 1] += eps * b * np.sin(a * X) * np.cos(b * Y) * np.sin(c * z)
    grad[:, 2] += eps * c * np.sin(a * X) * np.sin(b * Y) * np.cos(c * z)
    s = np.sqrt((grad * grad).sum(axis=1))
    s[src] = 1.0 / v0
    return StateCase(g, s, T, src)


def skew_box_grid(n, L=6.0, H=4.0, amp=0.4) -> Grid:
    """2-D convex box [0, L] x [0, H] with a non-orthogonal interior map (the boundary is
    mapped onto itself): x = xi + amp sin(pi zeta/H) sin(2 pi xi/L),
    z = zeta + amp/2 sin(pi xi/L) sin(2 pi zeta/H).  Straight and curved rays of a
    constant-gradient medium stay inside, so its closed form holds on the domain."""
    xi = np.linspace(0.0, L, n[0])
    ze = np.linspace(0.0, H, n[1])
    X, Z = np.meshgrid(xi, ze, indexing="ij")
    x = X + amp * np.sin(np.pi * Z / H) * np.sin(2 * np.pi * X / L)
    z = Z + 0.5 * amp * np.sin(np.pi * X / L) * np.sin(2 * np.pi * Z / H)
    xyz = np.ascontiguousarray(np.stack([x.ravel(), z.ravel()], axis=1))
    return Grid(2, tuple(n), (L / (n[0] - 1), H / (n[1] - 1)), xyz, (0.0, 0.0), H)


# ---------------------------------------------------------------------------
# Constant-gradient medium v = v0 + g z: closed-form first arrival
# ---------------------------------------------------------------------------
def linear_velocity_T(xyz: np.ndarray, xs: np.ndarray, v0: float, grad: float) -> np.ndarray:
    """First arrival in v(z) = v0 + grad*z from a point source at xs:
    T = arccosh(1 + grad^2 r^2 / (2 v(xs) v(x))) / grad (textbook closed form)."""
    d = xyz - xs
    r2 = (d * d).sum(axis=1)
    vs = v0 + grad * xs[-1]
    v = v0 + grad * xyz[:, -1]
    return np.arccosh(1.0 + grad * grad * r2 / (2.0 * vs * v)) / grad


# ---------------------------------------------------------------------------
# Topography and velocity recipes of the benchmark workloads
# ---------------------------------------------------------------------------
def gaussian_field_2d(nx: int, ny: int, dx: float, dy: float, corr: float, rms: float,
                      rng: np.random.Generator) -> np.ndarray:
    """Seeded smooth random surface: white noise filtered by a Gaussian spectrum
    exp(-k^2 corr^2 / 4) (correlation length corr), scaled to the given RMS."""
    w = rng.standard_normal((nx, ny))
    kx = 2 * np.pi * np.fft.fftfreq(nx, d=dx)
    ky = 2 * np.pi * np.fft.fftfreq(ny, d=dy)
    k2 = kx[:, None] ** 2 + ky[None, :] ** 2
    f = np.real(np.fft.ifft2(np.fft.fft2(w) * np.exp(-k2 * corr * corr / 4.0)))
    f -= f.mean()
    return f * (rms / np.sqrt((f * f).mean()))


@dataclass
class Workload:
    name: str
    grid: Grid
    s: np.ndarray             # [N] slowness
    src: np.ndarray           # [S] source node indices (surface nodes)
    rec: np.ndarray           # [n_rec] receiver node indices (shared by all sources)
    R: int                    # right-hand sides per source
    seed: int
    notes: dict = field(default_factory=dict)

    @property
    def S(self) -> int:
        return int(len(self.src))


def _surface_index(g: Grid, *h) -> int:
    return g.index(*h, 0)


def config1() -> Workload:
    """2-D, 61x41 over 6x4 km; elevation 0.4 sin(2 pi x/3) km; v = 1.5 + 0.5 z km/s with a
    +10% Gaussian anomaly (sigma 0.5 km) at (3, 2) km; 1 source at surface node 15,
    20 receivers at surface nodes 1 + 3k."""
    H = 4.0

    def zs(x):
        return -0.4 * np.sin(2 * np.pi * x / 3.0)

    g = mapped_grid((61, 41), (0.0,), (6.0,), H, zs)
    x, z = g.xyz[:, 0], g.xyz[:, 1]
    v = 1.5 + 0.5 * z
    v = v * (1.0 + 0.10 * np.exp(-((x - 3.0) ** 2 + (z - 2.0) ** 2) / (2 * 0.5 ** 2)))
    assert np.all(v > 0)
    src = np.array([_surface_index(g, 15)], dtype=np.int32)
    rec = np.array([_surface_index(g, 1 + 3 * k) for k in range(20)], dtype=np.int32)
    return Workload("2d-61x41-fp64", g, 1.0 / v, src, rec, 1, 20261)


def config2() -> Workload:
    """2-D, 401x201 over 20x10 km; three seeded Gaussian hills (height U(0.3, 1.5) km,
    slope U(20, 40) deg); v = 1.8 + 0.6 z with 8 seeded +-8% Gaussian anomalies;
    16 sources evenly spaced on the surface, 32 RHS each, 200 receivers (every 2nd node)."""
    seed = 20262
    rng = np.random.default_rng(seed)
    L, H = 20.0, 10.0
    cx = rng.uniform(0.15, 0.85, 3) * L
    hh = rng.uniform(0.3, 1.5, 3)
    th = np.deg2rad(rng.uniform(20.0, 40.0, 3))
    sig = hh / (math.sqrt(math.e) * np.tan(th))

    def elev(x):
        return sum(hh[m] * np.exp(-((x - cx[m]) ** 2) / (2 * sig[m] ** 2)) for m in range(3))

    g = mapped_grid((401, 201), (0.0,), (L,), H, lambda x: -elev(x))
    x, z = g.xyz[:, 0], g.xyz[:, 1]
    v = 1.8 + 0.6 * z
    ax = rng.uniform(0.0, L, 8)
    az = rng.uniform(0.5, H - 0.5, 8)
    asg = rng.uniform(0.5, 1.5, 8)
    amp = 0.08 * rng.choice([-1.0, 1.0], 8)
    fac = np.ones_like(v)
    for m in range(8):
        fac += amp[m] * np.exp(-((x - ax[m]) ** 2 + (z - az[m]) ** 2) / (2 * asg[m] ** 2))
    v = v * fac
    assert np.all(v > 0)
    src = np.array([_surface_index(g, int(round((k + 0.5) * 400 / 16))) for k in range(16)],
                   dtype=np.int32)
    rec = np.array([_surface_index(g, 2 * k) for k in range(200)], dtype=np.int32)
    xs = np.linspace(0, L, 4001)
    slope = np.degrees(np.arctan(np.abs(np.gradient(elev(xs), xs)).max()))
    return Workload("2d-401x201-batch", g, 1.0 / v, src, rec, 32, seed,
                    {"max_slope_deg": float(slope)})


def _config3d(name, n, Lxy, H, period, seed, hill_h=1.2, hill_sigma=3.0, rms=0.2, stride=1) -> Grid:
    """The 3-D recipe on an n grid; with stride > 1 the random surface is drawn on the grid
    refined stride times and sampled at every stride-th node, so the coarse grid's nodes
    lie on the fine grid's surface (a refinement pair of one model)."""
    rng = np.random.default_rng(seed)
    nx, ny = n[0], n[1]
    fx, fy = stride * (nx - 1) + 1, stride * (ny - 1) + 1
    field2 = gaussian_field_2d(fx, fy, Lxy / (fx - 1), Lxy / (fy - 1), 3.0, rms, rng)[::stride, ::stride]
    dx, dy = Lxy / (nx - 1), Lxy / (ny - 1)
    xc = yc = Lxy / 2

    def elev_grid():
        X, Y = np.meshgrid(np.arange(nx) * dx, np.arange(ny) * dy, indexing="ij")
        return hill_h * np.exp(-((X - xc) ** 2 + (Y - yc) ** 2) / (2 * hill_sigma ** 2)) + field2

    E = elev_grid()

    def zs(x, y):
        i = np.rint(x / dx).astype(np.int64)
        j = np.rint(y / dy).astype(np.int64)
        return -E[i, j]

    g = mapped_grid(n, (0.0, 0.0), (Lxy, Lxy), H, zs)
    gy, gx = np.gradient(E, dy, axis=1), np.gradient(E, dx, axis=0)
    slope = float(np.degrees(np.arctan(np.sqrt(gx ** 2 + gy ** 2).max())))
    return g, slope


def _velocity3d(g: Grid, period: float) -> np.ndarray:
    x, y, z = g.xyz[:, 0], g.xyz[:, 1], g.xyz[:, 2]
    v = 2.0 + 0.5 * z
    w = 2 * np.pi / period
    v = v * (1.0 + 0.05 * np.sin(w * x) * np.sin(w * y) * np.sin(w * z))
    assert np.all(v > 0)
    return v


def config3() -> Workload:
    """3-D, 101x101x51 over 20x20x8 km; 1.2 km Gaussian hill (sigma 3 km) on a seeded
    Gaussian-spectrum surface (correlation 3 km, RMS 0.2 km); v = 2.0 + 0.5 z with a
    +-5% smooth checkerboard of 2 km period; 25 sources at surface nodes {10,...,90}^2,
    64 RHS per source; receivers on the surface every 5th node (21 x 21)."""
    seed = 20263
    g, slope = _config3d("3d", (101, 101, 51), 20.0, 8.0, 2.0, seed)
    v = _velocity3d(g, 2.0)
    src = np.array([_surface_index(g, a, b) for a in (10, 30, 50, 70, 90) for b in (10, 30, 50, 70, 90)],
                   dtype=np.int32)
    rec = np.array([_surface_index(g, 5 * a, 5 * b) for a in range(21) for b in range(21)],
                   dtype=np.int32)
    return Workload("3d-101x101x51-S25-R64", g, 1.0 / v, src, rec, 64, seed,
                    {"max_slope_deg": slope})


def config4() -> Workload:
    """3-D, 201x201x101 over 40x40x15 km, same recipe with a 3 km checkerboard; 64 sources
    on an 8x8 surface lattice; 2500 receivers (50x50, every 4th surface node); 1 RHS."""
    seed = 20264
    g, slope = _config3d("3d", (201, 201, 101), 40.0, 15.0, 3.0, seed)
    v = _velocity3d(g, 3.0)
    lat = [12 + 25 * a for a in range(8)]
    src = np.array([_surface_index(g, a, b) for a in lat for b in lat], dtype=np.int32)
    rec = np.array([_surface_index(g, 4 * a + 2, 4 * b + 2) for a in range(50) for b in range(50)],
                   dtype=np.int32)
    return Workload("3d-201x201x101-S64-lsqr", g, 1.0 / v, src, rec, 1, seed,
                    {"max_slope_deg": slope})


def config4_refinement(level: int, nsrc: int = 4) -> Workload:
    """The config-4 model (201x201x101 over 40x40x15 km, 3 km checkerboard) at full size
    (level 1) or on the 101x101x51 grid whose nodes are every second node of it (level 0),
    with 4 sources and the 2500 receivers on nodes both grids share (the finite-difference
    check of the slowness -> traveltime function at two resolutions)."""
    seed = 20264
    stride = 1 if level == 1 else 2
    n = (201, 201, 101) if level == 1 else (101, 101, 51)
    g, slope = _config3d("3d", n, 40.0, 15.0, 3.0, seed, stride=stride)
    v = _velocity3d(g, 3.0)
    fine = [(12, 12), (62, 112), (112, 62), (162, 162)][:nsrc]
    src = np.array([_surface_index(g, a // stride, b // stride) for a, b in fine], dtype=np.int32)
    rec = np.array([_surface_index(g, (4 * a + 2) // stride, (4 * b + 2) // stride) for a in range(50) for b in range(50)],
                   dtype=np.int32)
    return Workload(f"3d-config4-model-{n[0]}x{n[1]}x{n[2]}", g, 1.0 / v, src, rec, 1, seed, {"max_slope_deg": slope})


def config5_grid(which: int) -> Workload:
    """One grid of the uneven-batch stress case: steep hill (slopes up to ~55 deg)."""
    seed = 20265 + which
    n, L, H, S, R = [((101, 101, 51), 20.0, 8.0, 32, 8),
                     ((161, 121, 61), 32.0, 10.0, 32, 32),
                     ((201, 201, 101), 40.0, 15.0, 64, 128)][which]
    hill_h = 1.2
    sig = hill_h / (math.sqrt(math.e) * math.tan(math.radians(55.0)))
    g, slope = _config3d("3d", n, L, H, 2.0, seed, hill_h=hill_h, hill_sigma=sig)
    v = _velocity3d(g, 2.0)
    na = 1 << int(math.floor(math.log2(math.sqrt(S))))   # lattice na x (S / na): 4 x 8 or 8 x 8
    ia = np.linspace(5, n[0] - 6, na).round().astype(int)
    ib = np.linspace(5, n[1] - 6, S // na).round().astype(int)
    src = np.array([_surface_index(g, a, b) for a in ia for b in ib], dtype=np.int32)
    rec = np.array([_surface_index(g, a, b) for a in range(2, n[0], 5) for b in range(2, n[1], 5)],
                   dtype=np.int32)
    return Workload(f"3d-stress-{which}", g, 1.0 / v, src, rec, R, seed, {"max_slope_deg": slope})


def rhs(shape, seed: int, dtype=np.float64) -> np.ndarray:
    """Seeded N(0, 1) right-hand sides."""
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)
