"""Seeded synthetic inputs for the LEM workloads (shared by the tests, the bench and the
oracle's callers; this module holds none of the method's arithmetic).

Every generator takes an explicit seed and uses numpy's PCG64. The workloads mirror the
paper's model problems (Eq. ibv / Eq. ibv2d: advection-diffusion with constant or variable
coefficients, Sec. 4) at the sizes the GPU path is built for:

* ``heat1d``      1D heat, N = 1024, Dirichlet, mu = nu dt / h^2 = 10, 16 tiles of 64, H = 16,
                  u0 = 8 sine modes with N(0, 1) amplitudes.
* ``advdiff2d``   2D periodic advection-diffusion, 2048^2, h = 1, dt = 4, nu = 5 (mu = 20),
                  velocity (1, 0.5) (C_x = 4, C_y = 2), first-order upwind + 5-point
                  Laplacian, tiles 32^2 + H = 8, u0 = Gaussian random field (length 16 h).
* ``vardiff2d``   2D Dirichlet diffusion-reaction div(k grad u) + u - u^3, 1024^2,
                  k = exp(GRF(32 h)) (lognormal, sigma = 1), tiles 16^2 + H = 6.
* ``vardiff1d``   1D Dirichlet diffusion (k u_x)_x, 2^20 nodes, lognormal k, median
                  diffusion number 2, tiles of 64 + H = 16 (a propagator per tile).

Stencil coefficients follow the C-ABI convention: entries of A (not dt-scaled) in the
order C, W, E, S, N, where W/E are the x - 1 / x + 1 neighbours and S/N the y - 1 / y + 1
neighbours of a row-major [y][x] mesh.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------- fields
def sine_modes_1d(n: int, nmodes: int, seed: int):
    """u0_j = sum_{k=1..nmodes} a_k sin(pi k j / (n + 1)), j = 1..n, a_k ~ N(0, 1)."""
    a = rng(seed).standard_normal(nmodes)
    j = np.arange(1, n + 1)
    u0 = np.zeros(n)
    for k in range(1, nmodes + 1):
        u0 += a[k - 1] * np.sin(np.pi * k * j / (n + 1))
    return u0, {k: float(a[k - 1]) for k in range(1, nmodes + 1)}


def grf_2d(shape, ell: float, seed: int, crop_from=None) -> np.ndarray:
    """Gaussian random field: white N(0,1) noise filtered by exp(-|kappa|^2 ell^2 / 4)
    in Fourier space, normalised to zero mean and unit standard deviation.
    ``crop_from`` generates on a larger periodic mesh and keeps the top-left corner
    (used for non-periodic problems)."""
    gshape = tuple(crop_from) if crop_from is not None else tuple(shape)
    w = rng(seed).standard_normal(gshape)
    ky = 2 * np.pi * np.fft.fftfreq(gshape[0])[:, None]
    kx = 2 * np.pi * np.fft.fftfreq(gshape[1])[None, :]
    filt = np.exp(-(kx ** 2 + ky ** 2) * ell ** 2 / 4.0)
    f = np.real(np.fft.ifft2(np.fft.fft2(w) * filt))
    f = f[: shape[0], : shape[1]]
    f = f - f.mean()
    return f / f.std()


def grf_1d(n: int, ell: float, seed: int) -> np.ndarray:
    w = rng(seed).standard_normal(n)
    k = 2 * np.pi * np.fft.fftfreq(n)
    f = np.real(np.fft.ifft(np.fft.fft(w) * np.exp(-k ** 2 * ell ** 2 / 4.0)))
    f = f - f.mean()
    return f / f.std()


# --------------------------------------------------------------------------- stencils
def stencil_heat_1d(nu: float, h: float) -> dict:
    """nu u_xx, centred: C = -2 nu/h^2, W = E = nu/h^2."""
    d = nu / h ** 2
    return {"C": -2 * d, "W": d, "E": d}


def stencil_advdiff_1d(nu: float, a: float, h: float, upwind: bool = False) -> dict:
    """-a u_x + nu u_xx: centred advection (Sec. 4 1D tests) or first-order upwind (a >= 0)."""
    d = nu / h ** 2
    if upwind:
        c = a / h
        return {"C": -2 * d - c, "W": d + c, "E": d}
    c = a / (2 * h)
    return {"C": -2 * d, "W": d + c, "E": d - c}


def stencil_advdiff_2d(nu: float, ax: float, ay: float, h: float) -> dict:
    """-a . grad u + nu Lap u with first-order upwind for a >= 0 and the 5-point Laplacian."""
    d = nu / h ** 2
    cx, cy = ax / h, ay / h
    return {"C": -4 * d - cx - cy, "W": d + cx, "E": d, "S": d + cy, "N": d}


def stencil_vardiff_1d(k: np.ndarray, h: float) -> dict:
    """(k u_x)_x with face coefficients k_{i+1/2} = (k_i + k_{i+1}) / 2; a face on a Dirichlet
    wall takes the value of its interior node. Returns per-node arrays."""
    kp = np.pad(k, (1, 1), mode="edge")
    W = 0.5 * (kp[1:-1] + kp[:-2]) / h ** 2
    E = 0.5 * (kp[1:-1] + kp[2:]) / h ** 2
    return {"C": -(W + E), "W": W, "E": E}


def stencil_vardiff_2d(k: np.ndarray, h: float) -> dict:
    """div(k grad u) with face coefficients k_{i+1/2} = (k_i + k_{i+1}) / 2; a face on a
    Dirichlet wall takes the value of its interior node. Returns per-node arrays."""
    kx = np.pad(k, ((0, 0), (1, 1)), mode="edge")
    ky = np.pad(k, ((1, 1), (0, 0)), mode="edge")
    W = 0.5 * (kx[:, 1:-1] + kx[:, :-2]) / h ** 2
    E = 0.5 * (kx[:, 1:-1] + kx[:, 2:]) / h ** 2
    S = 0.5 * (ky[1:-1, :] + ky[:-2, :]) / h ** 2
    N = 0.5 * (ky[1:-1, :] + ky[2:, :]) / h ** 2
    return {"C": -(W + E + S + N), "W": W, "E": E, "S": S, "N": N}


# --------------------------------------------------------------------------- workloads
def heat1d(n: int = 1024, tile: int = 64, overlap: int = 16, mu: float = 10.0,
           nmodes: int = 8, seed: int = 0) -> dict:
    h = 1.0 / (n + 1)
    nu = 1.0
    dt = mu * h ** 2 / nu
    u0, amps = sine_modes_1d(n, nmodes, seed)
    return dict(name=f"heat1d_N{n}", shape=(n,), bc=("dirichlet",),
                coef=stencil_heat_1d(nu, h), dt=dt, tile=(tile,), overlap=(overlap,),
                u0=u0, amps=amps, mu=mu, reaction=False)


def advdiff2d(side: int = 2048, tile=32, overlap=8, nu: float = 5.0,
              a=(1.0, 0.5), dt: float = 4.0, ell: float = 16.0, seed: int = 1) -> dict:
    """a = (a_x, a_y); h = 1, so mu = nu dt = 20 and (C_x, C_y) = dt a = (4, 2) by default.
    ``tile`` and ``overlap`` take one value for both axes or a (y, x) pair (anisotropic
    windows, e.g. a larger overlap along a fast vertical flow)."""
    coef = stencil_advdiff_2d(nu, a[0], a[1], 1.0)
    u0 = grf_2d((side, side), ell, seed).ravel()
    tile = (tile, tile) if np.isscalar(tile) else tuple(tile)
    overlap = (overlap, overlap) if np.isscalar(overlap) else tuple(overlap)
    return dict(name=f"advdiff2d_{side}", shape=(side, side), bc=("periodic", "periodic"),
                coef=coef, dt=dt, tile=tile, overlap=overlap, u0=u0, reaction=False)


def vardiff1d(n: int = 1 << 20, tile: int = 64, overlap: int = 16, mu_med: float = 2.0, ell_k: float = 32.0,
              sigma: float = 1.0, ell_u: float = 16.0, seed: int = 6) -> dict:
    """1D variable-coefficient diffusion (k u_x)_x, Dirichlet, k = exp(sigma GRF(ell_k h))
    (lognormal), dt from median(k) dt / h^2 = mu_med; u0 = GRF(ell_u h). Every window has its
    own local operator, so every tile has its own propagator (streamed from HBM each step)."""
    h = 1.0 / (n + 1)
    k = np.exp(sigma * grf_1d(n, ell_k, seed))
    dt = mu_med * h ** 2 / float(np.median(k))
    u0 = grf_1d(n, ell_u, seed + 100)
    return dict(name=f"vardiff1d_{n}", shape=(n,), bc=("dirichlet",), coef=stencil_vardiff_1d(k, h), dt=dt,
                tile=(tile,), overlap=(overlap,), u0=u0, reaction=False)


def vardiff2d(side: int = 1024, tile: int = 16, overlap: int = 6, ell_k: float = 32.0,
              sigma: float = 1.0, ell_u: float = 16.0, seed: int = 2) -> dict:
    """Variable-coefficient diffusion-reaction; dt from median(k) dt / h^2 = 2."""
    h = 1.0 / (side + 1)
    g = grf_2d((side, side), ell_k, seed, crop_from=(2 * side, 2 * side))
    k = np.exp(sigma * g)
    dt = 2.0 * h ** 2 / float(np.median(k))
    u0 = 0.5 * grf_2d((side, side), ell_u, seed + 100, crop_from=(2 * side, 2 * side))
    return dict(name=f"vardiff2d_{side}", shape=(side, side), bc=("dirichlet", "dirichlet"),
                coef=stencil_vardiff_2d(k, h), dt=dt, tile=(tile, tile),
                overlap=(overlap, overlap), u0=u0.ravel(), reaction=True)


def batch_problems(n: int = 512, seed: int = 3, side_max: int = 512) -> list:
    """Independent periodic 2D advection-diffusion problems of uneven size: side = 32 *
    U{2..side_max/32}, mu = nu dt / h^2 ~ U[1, 50], tile in {8, 16, 32}, overlap ~ U{4..8},
    C_x ~ U[0, 4] with C_y = C_x / 2 (h = 1, dt = 1), u0 = GRF(8)."""
    g = rng(seed)
    out = []
    for i in range(n):
        side = 32 * int(g.integers(2, side_max // 32 + 1))
        mu = float(g.uniform(1.0, 50.0))
        cx = float(g.uniform(0.0, 4.0))
        tile = int(g.choice([8, 16, 32]))
        H = int(g.integers(4, 9))
        coef = stencil_advdiff_2d(mu, cx, cx / 2, 1.0)
        u0 = grf_2d((side, side), 8.0, seed * 100000 + i).ravel()
        out.append(dict(name=f"batch{i}_{side}_t{tile}_H{H}", shape=(side, side), bc=("periodic", "periodic"),
                        coef=coef, dt=1.0, tile=(tile, tile), overlap=(H, H), u0=u0, reaction=False))
    return out


def schrodinger1d(n: int = 400, L: float = 10.0, kappa: float = 10.0, mu: float = 2.0, tile: int = 80,
                  overlap: int = 20, x0: float = -1.0, sigma: float = 0.5, seed: int = 5) -> dict:
    """1D Schroedinger equation with a harmonic potential, c_t = (i/2) c_xx - i (kappa/2) x^2 c,
    periodic on [-L/2, L/2) with n nodes, h = L / n, x_j = -L/2 + j h, centred second
    differences (Sec. 4.1). Complex stencil: C = -i/h^2 - i kappa x^2 / 2 (per node),
    W = E = i / (2 h^2). mu = dt / (2 h^2) is the stability parameter of the i/2 c_xx term, so
    dt = 2 mu h^2. u0 = a Gaussian of width sigma centred at x0 (real; seed unused, kept for a
    uniform generator signature)."""
    h = L / n
    x = -L / 2 + h * np.arange(n)
    coef = {"C": -1j / h ** 2 - 1j * kappa * x ** 2 / 2, "W": 1j / (2 * h ** 2) + 0 * x, "E": 1j / (2 * h ** 2) + 0 * x}
    u0 = np.exp(-(x - x0) ** 2 / (2 * sigma ** 2)).astype(np.complex128)
    return dict(name=f"schrodinger1d_{n}", shape=(n,), bc=("periodic",), coef=coef, dt=2 * mu * h * h,
                tile=(tile,), overlap=(overlap,), u0=u0, reaction=False, x=x, h=h)


def porous1d(n: int = 400, L: float = 10.0, m: float = 3.0, A: float = 1.0, t0: float = 1.0,
             mu: float = 4.0, tile: int = 40, overlap: int = 12, refresh: int = 1) -> dict:
    """1D porous-medium equation c_t = (c^m)_xx (Sec. 4.2, Eq. porous) on [-L/2, L/2] with
    homogeneous Dirichlet walls and n interior nodes, h = L / (n + 1), x_j = -L/2 + (j + 1) h,
    centred second differences applied to c^m (constant stencil C = -2/h^2, W = E = 1/h^2).
    u0 = the Barenblatt profile at time t0 (k = 1/(m+1)):
        t0^-k (A^2 - k (m-1) x^2 / (2 m t0^(2k)))_+^(1/(m-1)).
    dt = mu h^2 / max(m u0^(m-1)): mu is the stability parameter of the Jacobian's largest
    diffusivity at t0. The Jacobian is refreshed every ``refresh`` steps."""
    h = L / (n + 1)
    x = -L / 2 + h * (np.arange(n) + 1.0)
    k = 1.0 / (m + 1.0)
    u0 = t0 ** (-k) * np.maximum(A * A - k * (m - 1.0) * x * x / (2.0 * m * t0 ** (2.0 * k)), 0.0) ** (1.0 / (m - 1.0))
    dmax = m * float(np.max(np.abs(u0))) ** (m - 1.0)
    coef = {"C": -2.0 / h ** 2, "W": 1.0 / h ** 2, "E": 1.0 / h ** 2}
    return dict(name=f"porous1d_{n}", shape=(n,), bc=("dirichlet",), coef=coef, dt=mu * h * h / dmax,
                tile=(tile,), overlap=(overlap,), u0=u0, reaction=False, porous_m=m, refresh=refresh,
                x=x, h=h, t0=t0, A=A)
