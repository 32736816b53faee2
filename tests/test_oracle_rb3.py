"""Pins for phi_k and the third-order exponential Rosenbrock step (exprb32) of the oracle.

Sec. 2 defines the phi_k functions; Sec. 4.2 runs its nonlinear tests with a third-order
exponential Rosenbrock method (the scheme is not written out there; the reading is exprb32 of
Hochbruck, Ostermann and Schweitzer, 2009). Independent checks: phi_2 and phi_3 against their
closed forms in 50-digit arithmetic, the recurrence phi_k(X) = X phi_{k+1}(X) + I/k!, the
observed convergence order (3 for exprb32 against 2 for the exponential Euler-Rosenbrock step,
reference solution from an adaptive Runge-Kutta integrator), and reduction to the global step
when one window covers the mesh.
"""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import (assemble_operator, decompose, global_run, global_run_rb3, lem_run, lem_run_rb3, phi1, phik,
                    rb3_defect, rel_l2)
from paper_1505_02248_gb300 import workloads as W


@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("z", [-30.0, -4.0, -0.5, -1e-3, 0.0, 0.7, 2.5])
def test_phik_scalar_closed_form(k, z):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    zz = mp.mpf(z)
    if z == 0.0:
        ref = mp.mpf(1) / math.factorial(k)
    else:
        ref = (mp.e ** zz - sum(zz ** j / mp.factorial(j) for j in range(k))) / zz ** k
    got = phik(np.array([[z]]), k)[0, 0]
    assert abs(got - float(ref)) <= 1e-14 * max(1.0, abs(float(ref)))


def test_phik_recurrence_and_phi1():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((7, 7)) * 1.5
    for k in (1, 2):
        lhs = phik(X, k)
        rhs = X @ phik(X, k + 1) + np.eye(7) / math.factorial(k)
        assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(lhs).max()
    assert np.abs(phik(X, 1) - phi1(X)).max() <= 1e-13 * np.abs(phi1(X)).max()


def test_rb3_defect_is_pointwise_remainder():
    """dt (G(U) - G(u)) with G(v) = F(v) - J(u_m) v, evaluated through the full F and J."""
    rng = np.random.default_rng(6)
    n, dt = 12, 0.3
    Xg = assemble_operator((n,), ("dirichlet",), W.stencil_heat_1d(1.0, 1.0), dt)
    u, U, um = rng.standard_normal(n), rng.standard_normal(n), rng.standard_normal(n)
    F = lambda v: Xg @ v + dt * (v - v ** 3)                          # dt F(v)
    J = Xg.toarray() + np.diag(dt * (1.0 - 3.0 * um ** 2))            # dt J(u_m)
    ref = (F(U) - J @ U) - (F(u) - J @ u)
    assert np.abs(rb3_defect(u, U, um, dt) - ref).max() <= 1e-13


def _order(run, n=6, T=1.0):
    """Observed convergence order of a Rosenbrock run with the Jacobian refreshed every step,
    on u' = A u + u - u^3 (1D Dirichlet heat, 6 nodes)."""
    A = assemble_operator((n,), ("dirichlet",), W.stencil_heat_1d(1.0, 1.0 / (n + 1)), 1.0).toarray() / 50.0
    u0 = np.sin(np.pi * np.arange(1, n + 1) / (n + 1)) * 1.2
    ref = solve_ivp(lambda t, v: A @ v + v - v ** 3, (0, T), u0, method="DOP853", rtol=1e-13, atol=1e-14).y[:, -1]
    errs = []
    for m in (8, 16, 32):
        dt = T / m
        import scipy.sparse as sp
        Xg = sp.csr_matrix(A * dt)
        errs.append(np.abs(run(Xg, u0, m, dt) - ref).max())
    return [math.log2(errs[i] / errs[i + 1]) for i in range(2)]


def test_rb3_is_third_order_and_euler_second():
    p3 = _order(lambda Xg, u0, m, dt: global_run_rb3(Xg, u0, m, dt, refresh=1))
    p2 = _order(lambda Xg, u0, m, dt: global_run(Xg, u0, m, dt, True, refresh=1))
    assert all(2.7 < p < 3.3 for p in p3), p3
    assert all(1.7 < p < 2.3 for p in p2), p2


def test_rb3_one_window_is_global_step_and_overlap_helps():
    wl = W.vardiff2d(side=24, tile=8, overlap=3)
    Xg = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    one = decompose(wl["shape"], wl["bc"], (24, 24), (0, 0))
    g = global_run_rb3(Xg, wl["u0"], 4, wl["dt"], refresh=2)
    assert rel_l2(lem_run_rb3(Xg, wl["u0"], one, 4, wl["dt"], refresh=2), g) <= 1e-13
    e = [rel_l2(lem_run_rb3(Xg, wl["u0"], decompose(wl["shape"], wl["bc"], (8, 8), (H, H)), 4, wl["dt"],
                            refresh=2), g) for H in (1, 3, 6)]
    assert e[0] > e[1] > e[2]
