"""Pins for the oracle's decomposition and LEM step (Sec. 3, Eq. local_pb, Eq. lem).

Independent checks: the local problems solved by a general-purpose ODE integrator (the
definition of steps 1-3 of Sec. 3, with no matrix function at all), reduction to the
global method when one window covers the mesh, the paper's own qualitative statements on
buffer width (Sec. 4.1: Experiment 1 and Table 1), the shrinking of the LEM error with
overlap, and symmetries (linearity, translation equivariance).
"""
import os

import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import (assemble_operator, decompose, global_run, global_step, heat1d_dst_modes,
                    jacobian, lem_run, lem_step, local_propagators, phi1, rel_l2, residual)
from paper_1505_02248_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _kv(name):
    out = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


# --------------------------------------------------------------------------- decomposition
@pytest.mark.parametrize("shape,bc,tile,H", [
    ((1024,), ("dirichlet",), (64,), (16,)),
    ((100,), ("periodic",), (32,), (5,)),
    ((37, 45), ("dirichlet", "periodic"), (16, 16), (4, 6)),
    ((24, 24), ("periodic", "periodic"), (8, 8), (8, 8)),
])
def test_tiles_partition_mesh_and_windows_contain_tiles(shape, bc, tile, H):
    wins = decompose(shape, bc, tile, H)
    allD = np.concatenate([w.D for w in wins])
    assert np.array_equal(np.sort(allD), np.arange(int(np.prod(shape))))
    for w in wins:
        assert len(set(w.M.tolist())) == len(w.M)  # no node twice in a window
        assert np.array_equal(w.M[w.d_pos], w.D)


def test_heat1d_windows_are_clipped_at_walls():
    wins = decompose((1024,), ("dirichlet",), 64, 16)
    sizes = [len(w.M) for w in wins]
    assert len(wins) == 16 and sizes[0] == sizes[-1] == 80 and set(sizes[1:-1]) == {96}
    assert wins[0].M[0] == 0 and wins[-1].M[-1] == 1023


def test_periodic_windows_wrap():
    wins = decompose((64,), ("periodic",), 16, 4)
    assert wins[0].M.tolist() == list(range(60, 64)) + list(range(0, 20))
    assert wins[3].M.tolist() == list(range(44, 64)) + list(range(0, 4))


def test_ragged_last_tile():
    wins = decompose((70,), ("dirichlet",), 32, 3)
    assert [len(w.D) for w in wins] == [32, 32, 6]
    assert wins[2].M.tolist() == list(range(61, 70))


# --------------------------------------------------------------------------- local problems
def _local_ode_solution(Xg, u, w, mode):
    """Integrate the restricted problem of Eq. local_pb over one (dt-scaled) step.

    phi: Dirichlet data at the artificial boundary = neighbour values frozen at t^n,
         i.e. forcing g_M = (X u)|_M - X_M u|_M;  exp: zero data (g_M = 0)."""
    XM = Xg[w.M][:, w.M].toarray()
    g = (Xg @ u)[w.M] - XM @ u[w.M] if mode == "phi" else np.zeros(len(w.M))
    sol = solve_ivp(lambda t, v: XM @ v + g, (0.0, 1.0), u[w.M], method="DOP853",
                    rtol=1e-13, atol=1e-15)
    return sol.y[:, -1][w.d_pos]


@pytest.mark.parametrize("mode", ["phi", "exp"])
@pytest.mark.parametrize("case", ["1d_dirichlet_ragged", "2d_periodic", "2d_dirichlet_ragged"])
def test_lem_step_equals_local_ode_solutions(mode, case):
    rng = np.random.default_rng(42)
    if case == "1d_dirichlet_ragged":
        shape, bc, tile, H = (50,), ("dirichlet",), (16,), (5,)
        coef = W.stencil_advdiff_1d(1.0, 3.0, 1.0)
        dt = 2.0
    elif case == "2d_periodic":
        shape, bc, tile, H = (16, 16), ("periodic", "periodic"), (8, 8), (3, 3)
        coef = W.stencil_advdiff_2d(1.0, 1.0, 0.5, 1.0)
        dt = 1.5
    else:
        shape, bc, tile, H = (13, 11), ("dirichlet", "dirichlet"), (6, 4), (2, 3)
        coef = W.stencil_vardiff_2d(np.exp(rng.standard_normal((13, 11))), 1.0)
        dt = 0.7
    Xg = assemble_operator(shape, bc, coef, dt)
    u = rng.standard_normal(int(np.prod(shape)))
    wins = decompose(shape, bc, tile, H)
    props = local_propagators(Xg, wins, mode)
    got = lem_step(Xg, u, wins, props, mode)
    ref = u.copy()
    for w in wins:
        ref[w.D] = _local_ode_solution(Xg, u, w, mode)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("mode", ["phi", "exp"])
def test_one_window_covering_mesh_is_global_step(mode):
    wl = W.heat1d(n=96, mu=10.0)
    Xg = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], 32, 96)  # every window clips to the whole mesh
    assert all(len(w.M) == 96 for w in wins)
    u = lem_run(Xg, wl["u0"], wins, 5, mode)
    assert rel_l2(u, heat1d_dst_modes(96, 10.0, wl["amps"], 5)) < 1e-12


def test_periodic_whole_axis_window_is_global_step():
    wl = W.advdiff2d(side=16, ell=3.0, dt=0.5)  # mu = 2.5: the state stays O(1)
    Xg = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], 8, 4)  # 8 + 2*4 >= 16: whole axes
    assert all(len(w.M) == 256 for w in wins)
    assert rel_l2(lem_run(Xg, wl["u0"], wins, 3), global_run(Xg, wl["u0"], 3)) < 1e-12


def test_heat1d_lem_error_shrinks_with_overlap():
    wl = W.heat1d()
    Xg = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    ref = heat1d_dst_modes(1024, 10.0, wl["amps"], 100)
    errs = {}
    for H in (4, 8, 16, 24):
        wins = decompose(wl["shape"], wl["bc"], 64, H)
        errs[H] = rel_l2(lem_run(Xg, wl["u0"], wins, 100), ref)
    assert errs[4] > errs[8] > errs[16] > errs[24]
    assert errs[16] < 1e-5 and errs[24] < 1e-8


def test_lem_linearity_and_translation_equivariance():
    wl = W.advdiff2d(side=32, ell=4.0)
    Xg = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], 8, 4)
    props = local_propagators(Xg, wins, "phi")
    rng = np.random.default_rng(0)
    a, b = rng.standard_normal(1024), rng.standard_normal(1024)
    step = lambda v: lem_step(Xg, v, wins, props, "phi")
    assert np.allclose(step(2.0 * a - 3.0 * b), 2.0 * step(a) - 3.0 * step(b), atol=1e-12)
    shift = lambda v: np.roll(v.reshape(32, 32), (8, 16), axis=(0, 1)).ravel()
    assert np.allclose(step(shift(a)), shift(step(a)), atol=1e-12)


# --------------------------------------------------------------------------- the paper's statements
def _exp1(buffer, nsteps=None):
    p = _kv("paper_exp1_1d_advdiff.txt")
    n, L = int(p["npoints"]), p["L"]
    h = L / n
    dt = p["mu"] * h * h  # nu = 1
    a = p["courant"] * h / dt
    steps = int(round(p["T"] / dt)) if nsteps is None else nsteps
    coef = W.stencil_advdiff_1d(1.0, a, h)
    Xg = assemble_operator((n,), ("periodic",), coef, dt)
    x = h * np.arange(n)
    u0 = np.exp(-0.5 * ((x - L / 2) / (L / 20)) ** 2)
    tile = n // int(p["subdomains"])
    lem = lem_run(Xg, u0, decompose((n,), ("periodic",), tile, int(buffer)), steps)
    glob = global_run(Xg, u0, steps)
    k = 2 * np.pi * np.fft.fftfreq(n, d=h)
    pde = np.real(np.fft.ifft(np.fft.fft(u0) * np.exp((-1j * a * k - k * k) * steps * dt)))
    return lem, glob, pde


def test_paper_exp1_buffer18_matches_global_buffer5_fails():
    p = _kv("paper_exp1_1d_advdiff.txt")
    lem, glob, pde = _exp1(p["buffer_good"])
    e_glob, e_lem = rel_l2(glob, pde), rel_l2(lem, pde)
    assert rel_l2(lem, glob) < 0.05 * e_glob          # "essentially identical" errors
    assert abs(e_lem - e_glob) < 0.05 * e_glob
    lem5, _, _ = _exp1(p["buffer_bad"])
    assert rel_l2(lem5, glob) > 5 * e_glob            # "totally erroneous"


def test_paper_table1_buffers_keep_lem_close_to_global():
    rows = []
    with open(os.path.join(GOLD, "paper_table1_buffers.txt")) as f:
        for line in f:
            parts = line.split()
            if len(parts) == 3 and not line.startswith("#"):
                rows.append(tuple(float(x) for x in parts))
    assert len(rows) == 4
    n, L, T = 400, 10.0, 3.0
    h = L / n
    x = h * np.arange(n)
    u0 = np.exp(-0.5 * ((x - L / 2) / (L / 20)) ** 2)
    for C, mu, B in rows:
        dt = mu * h * h
        a = C * h / dt
        Xg = assemble_operator((n,), ("periodic",), W.stencil_advdiff_1d(1.0, a, h), dt)
        steps = int(round(T / dt))
        lem = lem_run(Xg, u0, decompose((n,), ("periodic",), n // 4, int(B)), steps)
        assert rel_l2(lem, global_run(Xg, u0, steps)) < 3e-3


# --------------------------------------------------------------------------- reaction (Rosenbrock)
def test_reaction_uniform_state_follows_scalar_exponential_euler():
    rng = np.random.default_rng(9)
    shape = (12, 12)
    k = np.exp(rng.standard_normal(shape))
    coef = W.stencil_vardiff_2d(k, 1.0)
    # periodic: the div-form stencil has zero row sums only with periodic face values
    kx = 0.5 * (k + np.roll(k, 1, axis=1)); kxe = 0.5 * (k + np.roll(k, -1, axis=1))
    ky = 0.5 * (k + np.roll(k, 1, axis=0)); kye = 0.5 * (k + np.roll(k, -1, axis=0))
    coef = {"W": kx, "E": kxe, "S": ky, "N": kye, "C": -(kx + kxe + ky + kye)}
    dt = 0.3
    Xg = assemble_operator(shape, ("periodic", "periodic"), coef, dt)
    for c in (0.4, -0.8, 1.3):
        u = np.full(144, c)
        z = dt * (1 - 3 * c * c)
        ref = c + (np.expm1(z) / z) * dt * (c - c ** 3)
        assert np.allclose(global_step(Xg, u, dt, reaction=True), ref, rtol=1e-12)
    assert np.array_equal(residual(Xg, np.zeros(144), dt, True), np.zeros(144))


def test_reaction_whole_window_lem_equals_global_rosenbrock():
    rng = np.random.default_rng(4)
    shape = (10, 10)
    coef = W.stencil_vardiff_2d(np.exp(0.5 * rng.standard_normal(shape)), 1.0)
    dt = 0.2
    Xg = assemble_operator(shape, ("dirichlet", "dirichlet"), coef, dt)
    u0 = 0.5 * rng.standard_normal(100)
    wins = decompose(shape, ("dirichlet", "dirichlet"), 5, 10)
    for R in (1, 2):
        a = lem_run(Xg, u0, wins, 4, "phi", dt, reaction=True, refresh=R)
        b = global_run(Xg, u0, 4, dt, reaction=True, refresh=R)
        assert rel_l2(a, b) < 1e-12
    # the frozen Jacobian matters: R = 1 and R = 4 differ
    c = lem_run(Xg, u0, wins, 4, "phi", dt, reaction=True, refresh=4)
    assert rel_l2(a, c) > 1e-8


def test_reaction_jacobian_is_derivative_of_residual():
    rng = np.random.default_rng(8)
    shape = (6, 7)
    Xg = assemble_operator(shape, ("dirichlet", "dirichlet"),
                           W.stencil_vardiff_2d(np.exp(rng.standard_normal(shape)), 1.0), 0.4)
    u = rng.standard_normal(42)
    J = jacobian(Xg, u, 0.4, True).toarray()
    eps = 1e-6
    for j in range(0, 42, 5):
        e = np.zeros(42); e[j] = eps
        fd = (residual(Xg, u + e, 0.4, True) - residual(Xg, u - e, 0.4, True)) / (2 * eps)
        assert np.allclose(J[:, j], fd, atol=1e-8)


def test_column_windows_win_at_high_vertical_courant_number():
    """Sec. 1 and Sec. 4.3: at a vertical Courant number far above the horizontal one, a
    decomposition into whole columns (overlap only across columns), or windows that extend
    further vertically, keeps LEM closer to the global step than square windows with more
    nodes. The same windows lose once the flow turns horizontal, so the gain comes from
    matching the overlap to the direction of transport. Reference: the periodic FFT step."""
    from oracle import periodic2d_fft_step
    side = 48
    u0 = W.grf_2d((side, side), 6.0, 7).ravel()
    cases = {"square": ((16, 16), (8, 8)), "tall": ((16, 16), (12, 4)), "columns": ((side, 8), (0, 4))}

    def errors(cx, cy):
        coef = W.stencil_advdiff_2d(2.0, cx, cy, 1.0)
        X = assemble_operator((side, side), ("periodic", "periodic"), coef, 1.0)
        ref = periodic2d_fft_step(u0.reshape(side, side), coef, 10).ravel()
        out = {}
        for k, (tile, H) in cases.items():
            wins = decompose((side, side), ("periodic", "periodic"), tile, H)
            out[k] = (rel_l2(lem_run(X, u0, wins, 10, "phi"), ref), max(len(w.M) for w in wins))
        return out

    v = errors(0.5, 6.0)
    assert v["tall"][1] < v["square"][1] and v["columns"][1] < v["square"][1]
    assert v["tall"][0] < v["square"][0] / 3 and v["columns"][0] < v["square"][0] / 2
    h = errors(6.0, 0.5)
    assert h["tall"][0] > 3 * h["square"][0] and h["columns"][0] > 3 * h["square"][0]
