"""Pins of the oracle's LSQR and of its model map M against mathematics outside the
oracle: SciPy's independent LSQR, the exact least-squares solution, the residual norm
that LSQR carries, and the scaling identity of Sec. 3.2 driven through J itself with
the velocity and relative-velocity model maps of Sec. 2.3."""
import numpy as np
import scipy.sparse.linalg as sla

from paper_2609_14982_b300 import workloads as W


def test_lsqr_matches_scipy_iterates_and_residual(oracle_mod):
    """After k steps the oracle's LSQR iterate equals scipy.sparse.linalg.lsqr's (no
    stopping tests), its phibar equals |b - A x_k|, and after n = 15 steps (exact
    arithmetic: the minimizer) it is numpy's least-squares solution."""
    rng = np.random.default_rng(1)
    A = rng.standard_normal((40, 15))
    b = rng.standard_normal(40)
    for k in (1, 2, 5, 15):
        x, phibar = oracle_mod.lsqr(lambda v: A @ v, lambda u: A.T @ u, b, k)
        xs = sla.lsqr(A, b, atol=0.0, btol=0.0, conlim=0.0, iter_lim=k)[0]
        assert np.max(np.abs(x - xs)) <= 1e-12 * np.max(np.abs(xs)), k
        assert abs(phibar - np.linalg.norm(b - A @ x)) <= 1e-12 * np.linalg.norm(b), k
    xe = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.max(np.abs(x - xe)) <= 1e-10 * np.max(np.abs(xe))


def test_lsqr_residual_decreases_and_sign_flip_is_caught(oracle_mod):
    """phibar = |b - A x_k| is nonincreasing (LSQR minimizes it over the Krylov space);
    an operator with a flipped transpose (a plausible sign slip) breaks the residual
    identity, so the identity above is a real check of the transpose."""
    rng = np.random.default_rng(2)
    A = rng.standard_normal((30, 12))
    b = rng.standard_normal(30)
    prev = np.inf
    for k in range(1, 13):
        x, phibar = oracle_mod.lsqr(lambda v: A @ v, lambda u: A.T @ u, b, k)
        assert phibar <= prev * (1 + 1e-12)
        prev = phibar
    xw, phw = oracle_mod.lsqr(lambda v: A @ v, lambda u: -(A.T @ u), b, 5)
    assert abs(phw - np.linalg.norm(b - A @ xw)) > 1e-3 * np.linalg.norm(b)


def _config1_tangent(O):
    wl = W.config1()
    g = wl.grid
    _, G, _ = O.metric(g)
    src = int(wl.src[0])
    v = 1.5 + 0.5 * g.xyz[:, 1]
    T = W.linear_velocity_T(g.xyz, g.xyz[src], 1.5, 0.5)
    s = 1.0 / v
    return g, s, v, T, O.build_tangent(g, G, T, s, src)


def test_model_maps_reproduce_the_scaling_identity_through_J(oracle_mod):
    """Sec. 2.3 / Sec. 3.2: a relative perturbation m = 1 (dv = v) is the slowness
    perturbation ds = -s, whose transported response is dT = -T exactly.  Driven through
    J with the relative model (p = 1) and with the velocity model (p = v); a wrong factor
    (for instance -s for the velocity model) gives a different ds and fails."""
    O = oracle_mod
    g, s, v, T, t = _config1_tangent(O)
    every = np.arange(g.N)
    Tn = np.linalg.norm(T)
    jr = O.J([t], s, every, np.ones((g.N, 1)), model=O.MODEL_RELATIVE)[0, :, 0]
    assert np.linalg.norm(jr + T) <= 1e-14 * Tn
    jv = O.J([t], s, every, v[:, None], model=O.MODEL_VELOCITY)[0, :, 0]
    assert np.linalg.norm(jv + T) <= 1e-14 * Tn
    # the same identity fails for the wrong velocity factor -s (ds = -1 instead of -s)
    wrong = O.solve(t, t.cs * (-s * v))
    assert np.linalg.norm(wrong + T) > 1e-2 * Tn
    # J^T of the same maps: <J p, y> = <p, J^T y> with y = e_k picks row k of J
    y = np.zeros((1, g.N, 1))
    k = g.N // 2
    y[0, k, 0] = 1.0
    for model, p in ((O.MODEL_RELATIVE, np.ones((g.N, 1))), (O.MODEL_VELOCITY, v[:, None])):
        row = O.JT([t], s, every, y, model=model)[:, 0]
        assert abs(row @ p[:, 0] + T[k]) <= 1e-13 * abs(T[k])


def test_model_factor_hand_values(oracle_mod):
    """ds for dv at three nodes, computed by hand: ds = -s^2 dv (velocity) and
    ds = -s m (relative), identity for slowness."""
    O = oracle_mod
    s = np.array([0.5, 0.25, 2.0])
    dv = np.array([1.0, 2.0, -0.5])
    assert np.array_equal(O.model_factor(s, O.MODEL_VELOCITY) * dv, np.array([-0.25, -0.125, 2.0]))
    assert np.array_equal(O.model_factor(s, O.MODEL_RELATIVE) * dv, np.array([-0.5, -0.5, 1.0]))
    assert np.array_equal(O.model_factor(s, O.MODEL_SLOWNESS) * dv, dv)
