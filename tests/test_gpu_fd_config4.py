"""GPU: the slowness -> receiver-traveltime autograd function on the config-4 model
(201 x 201 x 101 over 40 x 40 x 15 km, 2500 surface receivers) against central finite
differences (h = 1e-4 relative) of the state solve along 16 smooth random slowness
directions, at full size and on the 101 x 101 x 51 grid whose nodes are every second node
of it (2 sources, FP64 states converged to 1e-10, whose finite-difference noise at this h
is about 1e-6 relative; the objective is the sum of all receiver traveltimes).

The frozen tangent is discretized separately from the nonlinear state (Sec. 3.2), so it
is the derivative of the state solve only up to discretization error: the normwise
mismatch is reported at both resolutions and must shrink under refinement.  The
comparison uses the receivers' horizontal positions two nodes below the surface: the
state solver's boundary rule (a boundary node takes tau from its inward-diagonal
neighbour) makes surface traveltimes respond to the slowness one node inside, which the
calibrated upwind rows of the surface nodes do not follow; that surface layer's mismatch
is printed beside the result."""
import numpy as np
import pytest
import torch

from paper_2609_14982_b300 import eik
from paper_2609_14982_b300 import workloads as W
from paper_2609_14982_b300.autograd import slowness_to_traveltime

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _directions(g, k, seed):
    """k smooth random slowness directions (products of low-wavenumber sines with random
    wavenumbers 1..3 and phases), relative to the slowness."""
    rng = np.random.default_rng(seed)
    x, y, z = g.xyz[:, 0], g.xyz[:, 1], g.xyz[:, 2]
    out = []
    for _ in range(k):
        kx, ky, kz = rng.integers(1, 4, 3)
        px, py, pz = rng.uniform(0, 2 * np.pi, 3)
        out.append(np.sin(np.pi * kx * x / 40.0 + px) * np.sin(np.pi * ky * y / 40.0 + py) *
                   np.sin(np.pi * kz * (z + 2.0) / 17.0 + pz))
    return out


def _mismatch(level):
    wl = W.config4_refinement(level, nsrc=2)
    g = wl.grid
    dg = eik.DeviceGrid(g)
    s0 = torch.tensor(wl.s, device=DEV)
    srcs = [int(a) for a in wl.src]
    rec = np.asarray(wl.rec, dtype=np.int64) + 2          # two nodes below each surface receiver
    recd = torch.tensor(rec, device=DEV)
    surf = torch.tensor(np.asarray(wl.rec, dtype=np.int64), device=DEV)
    opts = eik.default_opts(eik_tol=1e-10)
    grads = []
    for r in (rec, np.asarray(wl.rec, dtype=np.int64)):
        s = s0.clone().requires_grad_(True)
        d = slowness_to_traveltime(s, dg, srcs, r.astype(np.int32), opts=opts)
        d.sum().backward()
        grads.append(s.grad)

    def f(sv):
        T, _ = eik.eik_forward(dg, sv, srcs, opts)
        return float(T[:, recd].sum()), float(T[:, surf].sum())

    h = 1e-4
    fds, lins, fds_s, lins_s = [], [], [], []
    for dv in _directions(g, 16, 11):
        dirv = torch.tensor(dv, device=DEV) * s0
        lins.append(float((grads[0] * dirv).sum()))
        lins_s.append(float((grads[1] * dirv).sum()))
        fp, fps = f(s0 + h * dirv)
        fm, fms = f(s0 - h * dirv)
        fds.append((fp - fm) / (2 * h))
        fds_s.append((fps - fms) / (2 * h))
    fds, lins, fds_s, lins_s = map(np.array, (fds, lins, fds_s, lins_s))
    return (float(np.linalg.norm(fds - lins) / np.linalg.norm(fds)),
            float(np.linalg.norm(fds_s - lins_s) / np.linalg.norm(fds_s)))


def test_fd_check_on_the_config4_model_at_two_resolutions():
    coarse, coarse_s = _mismatch(0)
    fine, fine_s = _mismatch(1)
    print(f"FD vs autograd normwise mismatch over 16 directions, receivers two nodes deep: "
          f"101x101x51 {coarse:.3e}, 201x201x101 {fine:.3e}; at the surface: {coarse_s:.3e}, {fine_s:.3e}")
    assert fine < coarse, (coarse, fine)
    assert fine < 0.1, (coarse, fine)
