"""Pins for the oracle's truncated propagators (Sec. 2, Theorem 1: entries of the
exponential of a banded matrix decay away from the band; the truncation keeps a box of
window nodes around each owner node).

Independent checks:
- closed forms. On a long periodic 1D mesh with the 3-point stencil X = W S_west + E S_east
  - (W + E) I (diffusion plus upwind advection), exp(X) is the transition kernel of a
  continuous-time random walk: exp(X)_{d, d+k} = e^{-(W+E)} (E/W)^{k/2} I_|k|(2 sqrt(E W))
  (I the modified Bessel function), and phi_1(X) is its integral over s in [0, 1]. A window
  much wider than the walk's spread reproduces them for its middle owner rows, so the
  offsets, the box and each side's extent can be predicted from the Bessel tails alone. In
  2D without advection the kernel is the product of two 1D kernels.
- tol = 0 keeps every nonzero entry (truncation is the identity).
- the triangle inequality: one truncated step moves every owner node by at most
  tol * max_d sum_m |P_dm| * max|r|.
"""
import numpy as np
import pytest
from scipy import integrate, special

from oracle import (assemble_operator, decompose, expm_pade13, local_propagators, lem_step, phi1,
                    residual, truncate_propagator, truncation_extents, window_offsets)
from paper_1505_02248_gb300 import workloads as W


def _walk_kernel(k, Wc, Ec, s=1.0):
    """exp(s X)_{d, d+k} for X = W S_west + E S_east - (W + E) I on the integer lattice."""
    k = np.asarray(k)
    z = 2.0 * s * np.sqrt(Wc * Ec)
    return np.exp(-s * (Wc + Ec) + z) * (Ec / Wc) ** (k / 2.0) * special.ive(np.abs(k), z)


def _walk_phi1(k, Wc, Ec):
    return np.array([integrate.quad(lambda s: _walk_kernel(kk, Wc, Ec, s), 0.0, 1.0,
                                    epsabs=1e-16, epsrel=1e-13)[0] for kk in np.atleast_1d(k)])


def _long_periodic_1d(mu, c, tile=16, H=40, n=512):
    coef = W.stencil_advdiff_1d(mu, c, 1.0, upwind=True)  # W = mu + c, E = mu, C = -(W + E)
    shape, bc = (n,), ("periodic",)
    X = assemble_operator(shape, bc, coef, 1.0)
    wins = decompose(shape, bc, (tile,), (H,))
    return coef, shape, X, wins


@pytest.mark.parametrize("mu,c", [(2.0, 0.0), (3.0, 1.5)])
def test_exp_and_phi1_rows_match_the_random_walk_kernel(mu, c):
    coef, shape, X, wins = _long_periodic_1d(mu, c)
    w = wins[0]
    XM = X[w.M][:, w.M].toarray()
    _, ox = window_offsets(w, shape)
    d = len(w.D) // 2  # a middle owner row: the window edges lie 48 nodes away
    E = expm_pade13(XM)[w.d_pos[d]]
    assert np.abs(E - _walk_kernel(ox[d], coef["W"], coef["E"])).max() <= 1e-13
    F = phi1(XM)[w.d_pos[d]]
    assert np.abs(F - _walk_phi1(ox[d], coef["W"], coef["E"])).max() <= 1e-13


@pytest.mark.parametrize("mu,c,tol", [(1.0, 0.0, 1e-8), (2.0, 1.0, 1e-8), (4.0, 2.0, 1e-10), (3.0, 0.0, 1e-6)])
def test_1d_extents_follow_from_the_kernel_tails(mu, c, tol):
    coef, shape, X, wins = _long_periodic_1d(mu, c)
    P = local_propagators(X, wins, "phi", tiles=[0])[0]
    ly, hy, lx, hx = truncation_extents(P, wins[0], shape, tol)
    assert ly == 0 and hy == 0
    # predicted from the lattice phi_1: row mass 1 (each exp(sX) row sums to one), each side's
    # smallest extent whose tail is within tol / 4
    k = np.arange(-60, 61)
    f = _walk_phi1(k, coef["W"], coef["E"])
    assert abs(f.sum() - 1.0) <= 1e-12

    def side(mask_of_e):
        e = 0
        while f[mask_of_e(e)].sum() > 0.25 * tol * f.sum():
            e += 1
        return e
    assert lx == side(lambda e: k < -e)
    assert hx == side(lambda e: k > e)
    if c > 0:
        assert lx > hx  # upwind advection carries the mass west of the owner


def test_2d_offsets_and_the_product_kernel():
    mu = 1.5
    coef = W.stencil_advdiff_2d(mu, 0.0, 0.0, 1.0)
    shape, bc = (48, 48), ("periodic", "periodic")
    X = assemble_operator(shape, bc, coef, 1.0)
    wins = decompose(shape, bc, (4, 4), (14, 14))  # 32 x 32 windows
    w = wins[0]
    oy, ox = window_offsets(w, shape)
    d = 5  # owner (1, 1) of the 4 x 4 tile, 15 nodes from every window edge
    E = expm_pade13(X[w.M][:, w.M].toarray())[w.d_pos[d]]
    g = lambda k: _walk_kernel(k, mu, mu)  # noqa: E731
    assert np.abs(E - g(oy[d]) * g(ox[d])).max() <= 1e-13
    # a window clipped at two walls (tile 0 of 8 x 8, H 4: window rows and columns 0..11):
    # offsets run from -7 (owner 7 to window node 0) to 11 (owner 0 to window node 11)
    wd = decompose((20, 20), ("dirichlet", "dirichlet"), (8, 8), (4, 4))[0]
    oyd, oxd = window_offsets(wd, (20, 20))
    assert (oyd.min(), oyd.max(), oxd.min(), oxd.max()) == (-7, 11, -7, 11)
    assert oyd[0, 0] == 0 and oxd[0, 13] == 1  # owner (0, 0) to window node (1, 1)


@pytest.mark.parametrize("case", ["1d_dirichlet", "2d_periodic_advection", "2d_dirichlet_vardiff"])
def test_zero_tolerance_keeps_every_entry(case):
    if case == "1d_dirichlet":
        wl = W.heat1d(n=256, tile=32, overlap=12, mu=3.0)
    elif case == "2d_periodic_advection":
        wl = W.advdiff2d(side=48, tile=8, overlap=6, nu=1.0, a=(2.0, 1.0), dt=1.0, ell=4.0)
    else:
        wl = W.vardiff2d(side=48, tile=16, overlap=6)
        wl["reaction"] = False
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    for t in (0, len(wins) // 2, len(wins) - 1):
        P = local_propagators(X, wins, "phi", tiles=[t])[t]
        ext = truncation_extents(P, wins[t], wl["shape"], 0.0)
        assert np.array_equal(truncate_propagator(P, wins[t], wl["shape"], ext), P)


@pytest.mark.parametrize("tol", [1e-4, 1e-6])
def test_one_truncated_step_moves_each_node_within_the_bound(tol):
    wl = W.advdiff2d(side=64, tile=16, overlap=8, nu=1.0, a=(2.0, 1.0), dt=1.0, ell=4.0)
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    props = local_propagators(X, wins, "phi")
    ext = truncation_extents(props[0], wins[0], wl["shape"], tol)
    assert ext[2] > ext[3] and ext[0] > ext[1]  # upwind: more kept upstream (west, south)
    assert max(ext) < 8 + 15  # something was dropped
    tprops = [truncate_propagator(P, w, wl["shape"], ext) for P, w in zip(props, wins)]
    u = wl["u0"]
    full = lem_step(X, u, wins, props, "phi")
    trunc = lem_step(X, u, wins, tprops, "phi")
    S = np.abs(props[0]).sum(axis=1).max()
    r = residual(X, u)
    assert np.abs(trunc - full).max() <= tol * S * np.abs(r).max()
    assert np.abs(trunc - full).max() > 0.0
