"""Planted mistakes in the oracle (on the CPU only): each plausible error below must make an
independent check fail, and the unmutated oracle must pass the same check. The checks rest on
closed forms, library routines or brute force, never on the oracle itself:

  expm: eigendecomposition of a symmetric matrix (numpy eigh)
  phi_1: the scalar closed form (e^z - 1) / z
  operator: the action on a plane wave (its symbol, C + W e^-ikh + E e^ikh)
  LEM: one window over the mesh equals exp(X) u (Sec. 2 identity)
  reaction: the scalar exponential-Euler step of c' = c - c^3 for a uniform state
  Jacobians: finite differences of the residual
  windows: the dilated, clipped tile listed by hand on a tiny mesh (Sec. 3, Fig. 3)
  porous medium: exact mass conservation of the global step (Sec. 4.2)
  Schroedinger: the free equation against its Fourier closed form (Sec. 4.1)
  phi_3: the scalar closed form (e^z - 1 - z - z^2/2) / z^3
  exprb32: the local error against a library ODE solver (scipy DOP853) falls by about 2^4
           per halving of dt (third order); a dropped factor 2 leaves about 2^3
  truncation: each side's extent against the one predicted from the Bessel tails of the 1D
           random-walk kernel (upwind advection makes the two sides differ); the window
           offsets of an anisotropic 2D window against their ranges worked out by hand
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy import integrate, special
from scipy.integrate import solve_ivp

import oracle.lem_oracle as OL
from paper_1505_02248_gb300 import workloads as W


def _heat(n=32, mu=10.0):
    return OL.assemble_operator((n,), ("dirichlet",), W.stencil_heat_1d(1.0, 1.0), mu).toarray()


def check_expm():
    X = _heat()
    lam, V = np.linalg.eigh(X)
    ref = (V * np.exp(lam)) @ V.T
    return np.abs(OL.expm_pade13(X) - ref).max() <= 1e-12 * np.abs(ref).max()


def check_phi1():
    z = np.array([[-3.7]])
    return abs(OL.phi1(z)[0, 0] - (np.exp(-3.7) - 1.0) / -3.7) <= 1e-14


def check_operator_symbol():
    n, h = 64, 1.0
    coef = {"C": -3.0, "W": 2.0, "E": 0.5}
    X = OL.assemble_operator((n,), ("periodic",), coef, 1.0)
    k = 2 * np.pi * 5 / n
    v = np.exp(1j * k * np.arange(n))
    lam = coef["C"] + coef["W"] * np.exp(-1j * k * h) + coef["E"] * np.exp(1j * k * h)
    return np.abs(X @ v - lam * v).max() <= 1e-12


def check_one_window_is_global():
    n = 40
    coef = {"C": -2.5, "W": 2.0, "E": 0.5}  # not symmetric: a transposed propagator shows
    X = OL.assemble_operator((n,), ("periodic",), coef, 0.8)
    u0 = np.sin(2 * np.pi * np.arange(n) / n) + 0.3 * np.cos(6 * np.pi * np.arange(n) / n)
    one = OL.decompose((n,), ("periodic",), (n,), (0,))
    got = OL.lem_run(X, u0, one, 3, "phi")
    lam, V = np.linalg.eig(X.toarray())
    ref = np.real(V @ np.diag(np.exp(3 * lam)) @ np.linalg.solve(V, u0))
    return OL.rel_l2(got, ref) <= 1e-12


def check_reaction_uniform_state():
    n, dt, c = 32, 0.3, 0.4
    X = OL.assemble_operator((n,), ("periodic",), W.stencil_heat_1d(1.0, 1.0), dt)
    got = OL.global_step(X, np.full(n, c), dt, True)
    z = dt * (1.0 - 3.0 * c * c)
    ref = c + (np.exp(z) - 1.0) / z * dt * (c - c ** 3)
    return np.abs(got - ref).max() <= 1e-13


def check_reaction_jacobian():
    n, dt = 24, 0.2
    X = OL.assemble_operator((n,), ("periodic",), W.stencil_heat_1d(1.0, 1.0), dt)
    rng = np.random.default_rng(3)
    u, v = rng.standard_normal(n), rng.standard_normal(n)
    eps = 1e-6
    fd = (OL.residual(X, u + eps * v, dt, True) - OL.residual(X, u - eps * v, dt, True)) / (2 * eps)
    return OL.rel_l2(OL.jacobian(X, u, dt, True) @ v, fd) <= 1e-8


def check_windows_by_hand():
    wins = OL.decompose((20,), ("dirichlet",), (5,), (3,))
    want = [list(range(0, 8)), list(range(2, 13)), list(range(7, 18)), list(range(12, 20))]
    return [w.M.tolist() for w in wins] == want


def check_porous_mass():
    wl = W.porous1d(n=60)
    X = OL.assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    g = OL.global_run(X, wl["u0"], 5, wl["dt"], refresh=1, porous_m=3.0)
    return abs(g.sum() / wl["u0"].sum() - 1.0) <= 1e-12


def check_free_schroedinger():
    wl = W.schrodinger1d(n=64, kappa=0.0, mu=2.0)
    X = OL.assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    got = OL.global_run(X, wl["u0"], 3)
    k = np.arange(64)
    lam = 0.5j * (-4.0 * np.sin(np.pi * k / 64) ** 2 / wl["h"] ** 2) * wl["dt"]
    ref = np.fft.ifft(np.fft.fft(wl["u0"]) * np.exp(3 * lam))
    return OL.rel_l2(got, ref) <= 1e-12


def check_phi3():
    z = -2.5
    ref = (np.exp(z) - 1.0 - z - z * z / 2.0) / z ** 3
    return abs(OL.phik(np.array([[z]]), 3)[0, 0] - ref) <= 1e-14


def check_rb3_local_order():
    n = 16
    coef = W.stencil_heat_1d(4.0, 1.0)
    A = OL.assemble_operator((n,), ("periodic",), coef, 1.0).toarray()
    u0 = 0.6 * np.sin(2 * np.pi * np.arange(n) / n) + 0.2
    errs = []
    for dt in (0.1, 0.05):
        X = OL.assemble_operator((n,), ("periodic",), coef, dt)
        exact = solve_ivp(lambda t, u: A @ u + u - u ** 3, (0.0, dt), u0, method="DOP853",
                          rtol=1e-13, atol=1e-14).y[:, -1]
        errs.append(np.linalg.norm(OL.global_step_rb3(X, u0, dt, u0.copy()) - exact))
    return errs[0] / errs[1] >= 10.0


def check_truncation_extents():
    # 1D periodic upwind advection-diffusion (W = mu + c, E = mu) on a long mesh: the window's
    # phi_1 rows follow the lattice random-walk kernel; predict each side's extent from it
    mu, c, tol = 2.0, 1.0, 1e-6  # (both sides move by one when tol is not split over them)
    n = 512
    coef = W.stencil_advdiff_1d(mu, c, 1.0, upwind=True)
    X = OL.assemble_operator((n,), ("periodic",), coef, 1.0)
    wins = OL.decompose((n,), ("periodic",), (16,), (40,))
    P = OL.local_propagators(X, wins, "phi", tiles=[0])[0]
    Wc, Ec = coef["W"], coef["E"]

    def kern(k, s):
        z = 2.0 * s * np.sqrt(Wc * Ec)
        return np.exp(-s * (Wc + Ec) + z) * (Ec / Wc) ** (k / 2.0) * special.ive(abs(k), z)
    ks = np.arange(-60, 61)
    f = np.array([integrate.quad(lambda s: kern(k, s), 0.0, 1.0, epsabs=1e-16, epsrel=1e-13)[0] for k in ks])

    def side(beyond):
        e = 0
        while f[beyond(e)].sum() > 0.25 * tol * f.sum():
            e += 1
        return e
    want = (0, 0, side(lambda e: ks < -e), side(lambda e: ks > e))
    return OL.truncation_extents(P, wins[0], (n,), tol) == want


def check_window_offsets_by_hand():
    # tile (4, 8) with H (6, 2) on a periodic 40 x 40 mesh: window 16 x 12, owners at window
    # rows 6..9 and columns 2..9; offsets run from -9 to 9 along y and from -9 to 9 along x,
    # but owner (0, 0) sees rows -6..9 and columns -2..9
    w = OL.decompose((40, 40), ("periodic", "periodic"), (4, 8), (6, 2))[0]
    oy, ox = OL.window_offsets(w, (40, 40))
    return (oy[0].min(), oy[0].max(), ox[0].min(), ox[0].max()) == (-6, 9, -2, 9) and oy.shape == (32, 192)


# ---------------------------------------------------------------- mutations
def m_drop_pade_term(mp):
    b = list(OL._B)
    b[5] = 0.0
    mp.setattr(OL, "_B", b)


def m_theta_too_large(mp):
    mp.setattr(OL, "THETA13", 60.0)


def m_swap_west_east(mp):
    orig = OL.assemble_operator

    def bad(shape, bc, coef, dt):
        c = dict(coef)
        c["W"], c["E"] = coef["E"], coef["W"]
        return orig(shape, bc, c, dt)
    mp.setattr(OL, "assemble_operator", bad)


def m_u_instead_of_r(mp):
    mp.setattr(OL, "residual", lambda Xg, u, dt=0.0, reaction=False, porous_m=0.0: u)


def m_transposed_propagator(mp):
    orig = OL.local_propagators
    mp.setattr(OL, "local_propagators", lambda *a, **k: [P.T.copy() if P is not None else None for P in orig(*a, **k)])


def m_phi1_is_exp(mp):
    mp.setattr(OL, "phi1", lambda X: OL.expm_pade13(X))


def m_reaction_sign(mp):
    orig = OL.residual

    def bad(Xg, u, dt=0.0, reaction=False, porous_m=0.0):
        return orig(Xg, u, dt, False, porous_m) + (dt * (u ** 3 - u) if reaction else 0.0)
    mp.setattr(OL, "residual", bad)


def m_reaction_jacobian(mp):
    orig = OL.jacobian

    def bad(Xg, u, dt, reaction, porous_m=0.0):
        if reaction and not porous_m:
            return (Xg + sp.diags(dt * (1.0 - u ** 2))).tocsr()
        return orig(Xg, u, dt, reaction, porous_m)
    mp.setattr(OL, "jacobian", bad)


def m_window_short_by_one(mp):
    orig = OL._axis_ranges

    def bad(n, tile, H, periodic):
        return [(d, w[1:] if len(w) > len(d) and w[0] != d[0] else w) for d, w in orig(n, tile, H, periodic)]
    mp.setattr(OL, "_axis_ranges", bad)


def m_porous_row_scaled(mp):
    orig = OL.jacobian

    def bad(Xg, u, dt, reaction, porous_m=0.0):
        if porous_m:
            return (sp.diags(porous_m * np.abs(u) ** (porous_m - 1.0)) @ Xg).tocsr()
        return orig(Xg, u, dt, reaction, porous_m)
    mp.setattr(OL, "jacobian", bad)


def m_conjugate_stencil(mp):
    orig = OL.assemble_operator
    mp.setattr(OL, "assemble_operator",
               lambda shape, bc, coef, dt: orig(shape, bc, {k: np.conj(v) for k, v in coef.items()}, dt))


def m_phik_off_by_one(mp):
    orig = OL.phik
    mp.setattr(OL, "phik", lambda X, k: orig(X, k - 1) if k == 3 else orig(X, k))


def m_rb3_factor_one(mp):
    orig = OL.rb3_defect
    mp.setattr(OL, "rb3_defect", lambda u, U, um, dt: 0.5 * orig(u, U, um, dt))


def m_trunc_sides_swapped(mp):
    orig = OL.truncation_extents

    def bad(P, window, shape, tol):
        ly, hy, lx, hx = orig(P, window, shape, tol)
        return (hy, ly, hx, lx)
    mp.setattr(OL, "truncation_extents", bad)


def m_trunc_whole_tol_per_side(mp):
    orig = OL.truncation_extents
    mp.setattr(OL, "truncation_extents", lambda P, window, shape, tol: orig(P, window, shape, 4.0 * tol))


def m_offsets_axes_swapped(mp):
    orig = OL.window_offsets

    def bad(window, shape):
        oy, ox = orig(window, shape)
        return ox, oy
    mp.setattr(OL, "window_offsets", bad)


CASES = {
    "dropped Pade term": (m_drop_pade_term, check_expm),
    "theta_13 too large": (m_theta_too_large, check_expm),
    "W and E swapped": (m_swap_west_east, check_operator_symbol),
    "u instead of the residual": (m_u_instead_of_r, check_one_window_is_global),
    "transposed propagator": (m_transposed_propagator, check_one_window_is_global),
    "phi_1 returns exp": (m_phi1_is_exp, check_phi1),
    "reaction sign flipped": (m_reaction_sign, check_reaction_uniform_state),
    "reaction Jacobian 1 - u^2": (m_reaction_jacobian, check_reaction_jacobian),
    "window short by one node": (m_window_short_by_one, check_windows_by_hand),
    "porous Jacobian row-scaled": (m_porous_row_scaled, check_porous_mass),
    "Schroedinger stencil conjugated": (m_conjugate_stencil, check_free_schroedinger),
    "phi_k one block off": (m_phik_off_by_one, check_phi3),
    "exprb32 correction factor 1": (m_rb3_factor_one, check_rb3_local_order),
    "truncation sides swapped": (m_trunc_sides_swapped, check_truncation_extents),
    "truncation tol not split over the sides": (m_trunc_whole_tol_per_side, check_truncation_extents),
    "window offsets with the axes swapped": (m_offsets_axes_swapped, check_window_offsets_by_hand),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_planted_mistake_is_caught(name, monkeypatch):
    mutate, check = CASES[name]
    assert check(), "the unmutated oracle must pass the check"
    mutate(monkeypatch)
    assert not check(), f"planted mistake '{name}' went unnoticed"
