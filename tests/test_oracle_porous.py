"""Pins for the oracle's porous-medium nonlinearity (Sec. 4.2, Eq. porous: c_t = (c^m)_xx).

The closed form (Barenblatt) is checked on its own first: it satisfies the PDE inside its
support and keeps its mass. The oracle is then held to it, and to properties a plausible
mistake breaks: the Jacobian is the derivative of the residual; the global exponential step
conserves mass exactly while the solution vanishes at the walls (X diag(phi'(u)) has zero
column sums there; diag(phi'(u)) X does not); one window over the mesh is the global step; the
LEM error shrinks with the buffer.
"""
import os

import numpy as np
import pytest

from oracle import (assemble_operator, barenblatt1d, decompose, global_run, jacobian, lem_run,
                    porous_phi, rel_l2, residual)
from paper_1505_02248_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _paper():
    kv = {}
    with open(os.path.join(GOLD, "paper_exp_porous.txt")) as f:
        for line in f:
            parts = line.split()
            if parts and not line.startswith("#"):
                kv[parts[0]] = float(parts[1])
    return kv


def _front(t, m, A):
    k = 1.0 / (m + 1.0)
    return A * np.sqrt(2.0 * m / (k * (m - 1.0))) * t ** k


def test_barenblatt_solves_the_pde_inside_its_support():
    p = _paper()
    m, A, t = p["m"], p["A"], 1.7
    x = np.linspace(-0.8, 0.8, 41) * _front(t, m, A)
    dt, dx = 1e-4, 1e-3
    ut = (barenblatt1d(x, t + dt, m, A) - barenblatt1d(x, t - dt, m, A)) / (2 * dt)
    um = lambda y: barenblatt1d(y, t, m, A) ** m  # noqa: E731
    uxx = (um(x + dx) - 2 * um(x) + um(x - dx)) / dx ** 2
    assert np.max(np.abs(ut - uxx)) <= 1e-5 * np.max(np.abs(ut))


def test_barenblatt_mass_is_constant_and_front_moves_as_t_to_the_k():
    p = _paper()
    m, A = p["m"], p["A"]
    masses = []
    for t in (1.0, 2.0, 4.0):
        xf = _front(t, m, A)
        x = np.linspace(-xf, xf, 400001)
        u = barenblatt1d(x, t, m, A)
        masses.append(np.trapezoid(u, x))
        # zero at the front (up to the square root of a rounding error) and beyond it
        assert max(u[0], u[-1]) <= 1e-7 and barenblatt1d(np.array([1.01 * xf]), t, m, A)[0] == 0.0
        assert barenblatt1d(np.array([0.99 * xf]), t, m, A)[0] > 0.0
    assert max(masses) - min(masses) <= 1e-6 * masses[0]


def test_porous_jacobian_is_derivative_of_residual():
    wl = W.porous1d(n=60)
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    rng = np.random.default_rng(11)
    u = rng.uniform(-0.5, 1.0, 60)
    v = rng.standard_normal(60)
    J = jacobian(X, u, wl["dt"], False, porous_m=3.0)
    eps = 1e-6
    fd = (residual(X, u + eps * v, wl["dt"], porous_m=3.0) - residual(X, u - eps * v, wl["dt"], porous_m=3.0)) / (2 * eps)
    assert rel_l2(J @ v, fd) <= 1e-8
    assert np.allclose(porous_phi(np.array([-2.0, 0.0, 0.5]), 3.0), [-8.0, 0.0, 0.125])


def test_global_step_follows_barenblatt_and_conserves_mass():
    p = _paper()
    wl = W.porous1d(n=100, L=p["L"], m=p["m"], A=p["A"])
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    steps = int(round(1.0 / wl["dt"]))
    g = global_run(X, wl["u0"], steps, wl["dt"], refresh=1, porous_m=p["m"])
    ref = barenblatt1d(wl["x"], wl["t0"] + steps * wl["dt"], p["m"], p["A"])
    assert rel_l2(g, ref) <= 2e-3                       # left alone, u0 is 0.25 away
    assert abs(g.sum() / wl["u0"].sum() - 1.0) <= 1e-12


def test_porous_lem_one_window_is_global_and_buffer_helps():
    wl = W.porous1d(n=100)
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    kw = dict(dt=wl["dt"], refresh=1, porous_m=3.0)
    one = lem_run(X, wl["u0"], decompose(wl["shape"], wl["bc"], (100,), (0,)), 10, **kw)
    assert rel_l2(one, global_run(X, wl["u0"], 10, **kw)) <= 1e-14
    steps = 40
    g = global_run(X, wl["u0"], steps, **kw)
    e = [rel_l2(lem_run(X, wl["u0"], decompose(wl["shape"], wl["bc"], (20,), (H,)), steps, **kw), g)
         for H in (2, 4, 8, 12)]
    assert e[0] > e[1] > e[2] > e[3] and e[3] <= 1e-7
