"""Pins for the oracle's operator assembly (Eq. spacedisc) and global exponential step.

Independent checks: eigenvalues of the 1D Dirichlet Laplacian (closed form), the Fourier
symbol of periodic stencils applied to plane waves, the drift (advection speed) and
spreading (diffusivity) of the exact semi-discrete solution, and mass conservation.
"""
import numpy as np
import pytest

from oracle import (assemble_operator, expm_pade13, global_run, global_step,
                    heat1d_dst_modes, heat1d_eigenvalues, periodic2d_fft_step,
                    periodic2d_symbol, rel_l2)
from paper_1505_02248_gb300 import workloads as W


def test_heat1d_eigenvalues_closed_form():
    n, mu = 50, 10.0
    X = assemble_operator((n,), ("dirichlet",), W.stencil_heat_1d(1.0, 1.0), mu).toarray()
    assert np.allclose(np.sort(np.linalg.eigvalsh(X)), np.sort(heat1d_eigenvalues(n, mu)),
                       rtol=1e-12, atol=1e-12)


def test_heat1d_global_step_vs_dst_modes():
    wl = W.heat1d(n=256, mu=10.0)
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    u = global_run(X, wl["u0"], 7)
    assert rel_l2(u, heat1d_dst_modes(256, 10.0, wl["amps"], 7)) < 1e-12


def test_dirichlet_walls_drop_outside_neighbours():
    coef = {"C": -4.0, "W": 1.0, "E": 2.0, "S": 3.0, "N": 5.0}
    X = assemble_operator((4, 5), ("dirichlet", "dirichlet"), coef, 1.0)
    rs = np.asarray(X.sum(axis=1)).reshape(4, 5)
    assert rs[0, 0] == -4 + 2 + 5          # corner (y=0, x=0): no W, no S
    assert rs[3, 4] == -4 + 1 + 3          # corner (y=3, x=4): no E, no N
    assert rs[2, 2] == -4 + 1 + 2 + 3 + 5  # interior
    assert X[7, 6] == 1.0 and X[7, 8] == 2.0 and X[7, 2] == 3.0 and X[7, 12] == 5.0


@pytest.mark.parametrize("shape", [(6, 8), (9, 7)])
def test_periodic_stencil_acts_by_its_symbol_on_plane_waves(shape):
    coef = {"C": -7.0, "W": 2.5, "E": 1.5, "S": 1.25, "N": 0.75}
    X = assemble_operator(shape, ("periodic", "periodic"), coef, 1.0)
    ny, nx = shape
    lam = periodic2d_symbol(shape, coef)
    for ky in range(ny):
        for kx in range(nx):
            y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
            wave = np.exp(2j * np.pi * (kx * x / nx + ky * y / ny)).ravel()
            assert np.allclose(X @ wave, lam[ky, kx] * wave, atol=1e-12)


def test_fft_step_vs_dense_expm():
    wl = W.advdiff2d(side=12, ell=2.0, dt=0.25)  # mu = 1.25: the state stays O(1)
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    u0 = wl["u0"]
    cdt = {k: v * wl["dt"] for k, v in wl["coef"].items()}
    ref = periodic2d_fft_step(u0.reshape(12, 12), cdt, 3).ravel()
    assert rel_l2(global_run(X, u0, 3), ref) < 1e-12


def test_upwind_advection_moves_mass_by_courant_number():
    # pure advection, first-order upwind, periodic: the exact semi-discrete solution's
    # centre of mass moves by C = a dt / h per step in +x (the Poisson-process mean).
    n, C = 512, 4.0
    coef = W.stencil_advdiff_1d(0.0, 1.0, 1.0, upwind=True)
    X = assemble_operator((n,), ("periodic",), coef, C)
    x = np.arange(n, dtype=float)
    u0 = np.exp(-0.5 * ((x - 200.0) / 6.0) ** 2)
    u1 = global_step(X, u0)
    com = lambda u: (x * u).sum() / u.sum()
    assert com(u1) - com(u0) == pytest.approx(C, abs=1e-9)
    assert u1.sum() == pytest.approx(u0.sum(), rel=1e-13)


def test_diffusion_spreads_variance_by_two_mu_per_step():
    n, mu = 600, 20.0
    X = assemble_operator((n,), ("periodic",), W.stencil_heat_1d(1.0, 1.0), mu)
    x = np.arange(n, dtype=float)
    u0 = np.exp(-0.5 * ((x - 300.0) / 8.0) ** 2)
    u1 = global_step(X, u0)
    var = lambda u: ((x - (x * u).sum() / u.sum()) ** 2 * u).sum() / u.sum()
    assert var(u1) - var(u0) == pytest.approx(2 * mu, rel=1e-9)


def test_global_periodic_step_conserves_mass():
    wl = W.advdiff2d(side=16, ell=3.0)
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    E = expm_pade13(X.toarray())
    assert np.allclose(E.sum(axis=0), 1.0, atol=1e-12)
    u1 = global_run(X, wl["u0"], 5)
    assert u1.sum() == pytest.approx(wl["u0"].sum(), abs=1e-10)
