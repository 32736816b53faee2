"""Plain FP64 statement of the Local Exponential Method (LEM), arXiv 1505.02248.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; never by the product path.

What is here, in the paper's order and notation (dt-scaled throughout, X = dt*A):

* ``assemble_operator`` -- the sparse matrix A of the semi-discrete system
  du/dt = A u + g (Eq. spacedisc, Sec. 2) from a 3-point (1D) or 5-point (2D) stencil.
  Homogeneous Dirichlet walls drop the outside neighbour (g = 0, Sec. 3: the mesh holds
  interior nodes only); periodic axes wrap.
* ``decompose`` -- the overlapping decomposition M_i = D_i U B_i (Sec. 3, Fig. 3): owner
  tiles D_i partition the mesh, windows M_i dilate them by the buffer width H per side,
  clipped at walls, wrapped on periodic axes.
* ``expm_pade13`` -- exp(X) by diagonal Pade approximation with scaling and squaring
  (Sec. 1 and Sec. 4 name the method; the degree 13 / theta_13 choice is Higham's 2005
  algorithm, stated here as a reading because the paper gives no degree or norm rule).
* ``phi1`` -- phi_1(X) = (e^X - I) X^{-1} (Sec. 2, phi_k definition with the sum to k-1),
  taken as the top-right block of exp([[X, I], [0, 0]]); ``phik`` the same for any k.
* ``local_propagators`` / ``lem_step`` -- the LEM exponential-Euler step (Eq. lem and
  steps 1-3 of Sec. 3): each window advances its restricted problem (Eq. local_pb) and only
  the owner rows D_i are written back. Two readings of the artificial-boundary data:
  ``phi`` (neighbour values frozen at t^n, the literal Eq. lem) and ``exp`` (zero data).
* ``global_step`` -- the global exponential-Euler step the LEM approximates
  (variation-of-constants identity, Sec. 2), by dense matrices (small N),
  ``heat1d_dst_modes`` (1D Dirichlet Laplacian, closed form) and ``periodic2d_fft_step``
  (constant-coefficient periodic 2D operator, closed form via its Fourier symbol).

* ``lem_step_rb3`` / ``lem_run_rb3`` -- a third-order exponential Rosenbrock step in LEM
  form. Sec. 4.2 runs its nonlinear tests with a third-order exponential Rosenbrock method
  without writing it out; the scheme taken is exprb32 (Hochbruck, Ostermann and Schweitzer,
  2009): a phi_1 stage and a phi_3 correction, both applied window by window.
  ``global_step_rb3`` / ``global_run_rb3`` are the same scheme on the whole mesh.

* ``window_offsets`` / ``truncation_extents`` / ``truncate_propagator`` -- truncated
  propagators. Sec. 2 (Theorem 1, after Iserles) states that the entries of the exponential
  of a banded matrix decay faster than exponentially away from the band; that decay is why
  the local problems work at all. A truncated propagator keeps, for every owner row, only
  the window nodes inside a box around the owner node (offsets -ly..hy along y, -lx..hx
  along x in window coordinates) and zeroes the rest. Each side's extent is the smallest
  whose dropped mass, max over rows of sum |P| beyond it, is at most tol/4 of the largest
  row mass max_d sum_m |P_dm|; the four sides together then drop at most tol of it. The
  tolerance rule is a reading: the paper gives no truncation rule.

* ``porous_m`` (``residual``, ``jacobian``, the step and run functions) -- the porous-medium
  equation c_t = (c^m)_xx of Sec. 4.2 (Eq. porous): dt F(u) = X phi(u), dt F'(u) =
  X diag(phi'(u)) with phi(u) = |u|^(m-1) u; ``barenblatt1d`` its closed-form solution.

Parity status: every function above is pinned in ``tests/test_oracle_*.py``.
The reaction (u - u^3) Rosenbrock variant is pinned only by invariants and by agreement
with the global step as H grows (no closed form exists for it).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from fractions import Fraction

import numpy as np
import scipy.sparse as sp

__all__ = [
    "THETA13", "pade13_coefficients", "squaring_count", "expm_pade13", "phi1", "phik",
    "assemble_operator", "Window", "decompose", "local_propagators", "residual",
    "jacobian", "lem_step", "lem_run", "global_step", "global_run",
    "rb3_defect", "lem_step_rb3", "lem_run_rb3", "global_step_rb3", "global_run_rb3",
    "porous_phi", "barenblatt1d", "heat1d_dst_modes", "heat1d_eigenvalues", "periodic2d_symbol", "periodic2d_fft_step",
    "window_offsets", "truncation_extents", "truncate_propagator",
    "rel_l2",
]

# theta_13 of Higham (2005), "The scaling and squaring method for the matrix exponential
# revisited", Table 2.3: the largest 1-norm for which degree-13 Pade meets unit roundoff.
THETA13 = 5.371920351148152
PADE_DEGREE = 13


def _fp(x) -> np.ndarray:
    """x as FP64, real or complex (complex problems, e.g. the Schroedinger test of Sec. 4.1,
    run through the same functions)."""
    x = np.asarray(x)
    return x.astype(np.complex128 if np.iscomplexobj(x) else np.float64)


def pade13_coefficients(m: int = PADE_DEGREE) -> list[float]:
    """Coefficients b_j of the numerator p_m(x) = sum_j b_j x^j of the [m/m] Pade
    approximant to e^x; the denominator is p_m(-x). (Sec. 1 and Sec. 4 name Pade
    approximation with scaling and squaring; m = 13 follows Higham 2005.)

    b_j = (2m - j)! m! / ((2m)! j! (m - j)!), computed exactly as rationals then rounded.
    """
    f = math.factorial
    return [float(Fraction(f(2 * m - j) * f(m), f(2 * m) * f(j) * f(m - j))) for j in range(m + 1)]


_B = pade13_coefficients()


def squaring_count(norm1: float) -> int:
    """Smallest s >= 0 with norm1 / 2^s <= theta_13 (exact 1-norm, no estimate): the scaling
    step of the scaling-and-squaring method named in Sec. 1 and Sec. 4 (Higham 2005's rule)."""
    s = 0
    while norm1 > THETA13 * (2.0 ** s):
        s += 1
    return s


def expm_pade13(X: np.ndarray) -> np.ndarray:
    """exp(X) by degree-13 Pade approximation with scaling and squaring (the method Sec. 1
    and Sec. 4 name for the local matrix exponentials; Higham 2005's degree and theta).

    1. s from the exact 1-norm (``squaring_count``); 2. scale X by 2^-s;
    3. U (odd part) and V (even part) of p_13 from X^2, X^4, X^6;
    4. solve (V - U) R = (V + U); 5. square R s times.
    """
    X = _fp(X)
    n = X.shape[0]
    s = squaring_count(float(np.abs(X).sum(axis=0).max()) if n else 0.0)
    X = X / (2.0 ** s)
    b = _B
    ident = np.eye(n)
    X2 = X @ X
    X4 = X2 @ X2
    X6 = X4 @ X2
    U = X @ (X6 @ (b[13] * X6 + b[11] * X4 + b[9] * X2)
             + b[7] * X6 + b[5] * X4 + b[3] * X2 + b[1] * ident)
    V = (X6 @ (b[12] * X6 + b[10] * X4 + b[8] * X2)
         + b[6] * X6 + b[4] * X4 + b[2] * X2 + b[0] * ident)
    R = np.linalg.solve(V - U, V + U)
    for _ in range(s):
        R = R @ R
    return R


def phi1(X: np.ndarray) -> np.ndarray:
    """phi_1(X) = sum_k X^k / (k+1)! (Sec. 2, phi_k with k = 1; the matrix function of Eq. lem):
    the top-right block of exp([[X, I], [0, 0]])."""
    X = _fp(X)
    n = X.shape[0]
    Z = np.zeros((2 * n, 2 * n), dtype=X.dtype)
    Z[:n, :n] = X
    Z[:n, n:] = np.eye(n)
    return expm_pade13(Z)[:n, n:]


def phik(X: np.ndarray, k: int) -> np.ndarray:
    """phi_k(X) = sum_j X^j / (j + k)! (Sec. 2 phi_k, sum to k - 1): the top-right block of
    exp(Z), Z the (k + 1) x (k + 1) block matrix with X in the top-left corner, identity
    blocks on the first block superdiagonal and zeros elsewhere (the top block row of exp(Z)
    is e^X, phi_1(X), ..., phi_k(X))."""
    X = _fp(X)
    n = X.shape[0]
    Z = np.zeros(((k + 1) * n, (k + 1) * n), dtype=X.dtype)
    Z[:n, :n] = X
    for j in range(k):
        Z[j * n:(j + 1) * n, (j + 1) * n:(j + 2) * n] = np.eye(n)
    return expm_pade13(Z)[:n, k * n:]


# --------------------------------------------------------------------------- operator
def _as_field(v, shape):
    """A stencil coefficient of Eq. spacedisc as a field over the mesh (scalars broadcast)."""
    a = _fp(v)
    return np.broadcast_to(a, shape) if a.ndim == 0 else a.reshape(shape)


def assemble_operator(shape, bc, coef, dt: float) -> sp.csr_matrix:
    """dt * A for the stencil ``coef`` on a ``shape`` mesh (Eq. spacedisc).

    Row p (flat row-major index, x = last axis) of A:
        A[p, p] = C_p,  A[p, p - e_x] = W_p,  A[p, p + e_x] = E_p,
        A[p, p - e_y] = S_p,  A[p, p + e_y] = N_p          (2D only for S, N).
    ``coef`` values are scalars (constant coefficients) or arrays of ``shape``.
    ``bc[axis]`` is 'dirichlet' (outside neighbours dropped: homogeneous data, g = 0)
    or 'periodic' (indices wrap).
    """
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    npts = int(np.prod(shape))
    idx = np.arange(npts).reshape(shape)
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [_as_field(coef["C"], shape).ravel()]
    # (name, axis, offset): W/E along x (last axis), S/N along y (first axis of a 2D mesh)
    nbrs = [("W", nd - 1, -1), ("E", nd - 1, +1)]
    if nd == 2:
        nbrs += [("S", 0, -1), ("N", 0, +1)]
    for name, axis, off in nbrs:
        c = _as_field(coef[name], shape)
        pos = np.indices(shape)
        q = pos[axis] + off
        n = shape[axis]
        if bc[axis] == "periodic":
            q = q % n
            keep = np.ones(shape, dtype=bool)
        else:
            keep = (q >= 0) & (q < n)
        pos[axis] = np.where(keep, q, 0)
        nb = np.ravel_multi_index(tuple(pos), shape)
        rows.append(idx[keep])
        cols.append(nb[keep])
        vals.append(c[keep])
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(npts, npts)).tocsr()  # duplicate entries (tiny periodic axes) add
    return (dt * A).tocsr()


# --------------------------------------------------------------------------- decomposition
@dataclass
class Window:
    """One subdomain: owner nodes D (global flat indices, row-major), window nodes M
    (global flat indices in window row-major order) and the positions of D inside M."""
    D: np.ndarray
    M: np.ndarray
    d_pos: np.ndarray


def _axis_ranges(n: int, tile: int, H: int, periodic: bool):
    """Along one axis: each tile's owner nodes and its window, the tile dilated by H per side
    (Sec. 3, Fig. 3), clipped at a wall or wrapped on a periodic axis."""
    out = []
    for t0 in range(0, n, tile):
        t1 = min(t0 + tile, n)  # the last tile may be ragged
        if periodic:
            if (t1 - t0) + 2 * H >= n:
                win = list(range(n))  # the window covers the whole periodic axis
            else:
                win = [(k % n) for k in range(t0 - H, t1 + H)]
        else:
            win = list(range(max(0, t0 - H), min(n, t1 + H)))  # clipped at the wall
        out.append((list(range(t0, t1)), win))
    return out


def decompose(shape, bc, tile, overlap) -> list[Window]:
    """Owner tiles D_i and windows M_i = D_i dilated by H per side (Sec. 3, Fig. 3).

    ``tile`` and ``overlap`` are per-axis (or scalars). Tiles are ordered row-major over
    the tile grid. Windows are clipped at Dirichlet walls (no node exists beyond the mesh)
    and wrapped on periodic axes; a periodic window that would reach around the whole axis
    is the whole axis in natural order.
    """
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    tile = (tile,) * nd if np.isscalar(tile) else tuple(tile)
    overlap = (overlap,) * nd if np.isscalar(overlap) else tuple(overlap)
    per_axis = [_axis_ranges(shape[a], tile[a], overlap[a], bc[a] == "periodic") for a in range(nd)]
    wins = []
    if nd == 1:
        for dx, mx in per_axis[0]:
            D = np.array(dx)
            M = np.array(mx)
            pos = {g: k for k, g in enumerate(mx)}
            wins.append(Window(D, M, np.array([pos[g] for g in dx])))
        return wins
    ny, nx = shape
    for dy, my in per_axis[0]:
        for dx, mx in per_axis[1]:
            D = np.array([y * nx + x for y in dy for x in dx])
            M = np.array([y * nx + x for y in my for x in mx])
            pos = {g: k for k, g in enumerate(M.tolist())}
            wins.append(Window(D, M, np.array([pos[g] for g in D.tolist()])))
    return wins


# --------------------------------------------------------------------------- LEM
def local_propagators(Xg: sp.csr_matrix, windows, mode: str = "phi", tiles=None):
    """P_i = R_{D_i} f(X_{M_i}) for every window (Eq. lem, steps 1-2 of Sec. 3).

    X_{M_i} is the principal submatrix of the dt-scaled global operator on M_i (the
    restriction with Dirichlet conditions at the artificial boundary). f = phi_1 for
    mode 'phi' (the step applies it to the dt-scaled residual), f = phi_3 for mode 'phi3'
    (the correction stage of the third-order Rosenbrock step) and f = exp for mode 'exp'.
    Windows with identical local matrices reuse one result (memoisation only).
    ``tiles`` restricts the work to a subset of window indices (others are None).
    """
    cache = {}
    out = [None] * len(windows)
    sel = range(len(windows)) if tiles is None else tiles
    for i in sel:
        w = windows[i]
        XM = Xg[w.M][:, w.M].tocsr()
        XM.sort_indices()
        key = (XM.shape, XM.indptr.tobytes(), XM.indices.tobytes(), XM.data.tobytes(),
               w.d_pos.tobytes())
        if key not in cache:
            if mode == "phi":
                F = phi1(XM.toarray())
            elif mode == "phi3":
                F = phik(XM.toarray(), 3)
            else:
                F = expm_pade13(XM.toarray())
            cache[key] = F[w.d_pos, :]
        out[i] = cache[key]
    return out


# --------------------------------------------------------------------------- truncation
def window_offsets(window: Window, shape):
    """(oy, ox): for every owner row d and window node m, the offset of m from the owner node
    d in window coordinates (window rows and columns, row-major order of M), each an
    n_int x n_loc integer array. 1D problems have oy = 0."""
    shape = tuple(int(s) for s in shape)
    nloc = len(window.M)
    if len(shape) == 1:
        wx = nloc
    else:
        wx = len(np.unique(window.M % shape[1]))
    k = np.arange(nloc)
    cy, cx = k // wx, k % wx
    dy, dx = cy[window.d_pos], cx[window.d_pos]
    return cy[None, :] - dy[:, None], cx[None, :] - dx[:, None]


def truncation_extents(P: np.ndarray, window: Window, shape, tol: float):
    """(ly, hy, lx, hx): the box a truncated propagator keeps (Sec. 2, Theorem 1: off-band
    decay). For each side, e.g. x below the owner, the smallest extent e >= 0 such that
    max_d sum_{m : ox_dm < -e} |P_dm| <= (tol / 4) * max_d sum_m |P_dm|."""
    oy, ox = window_offsets(window, shape)
    A = np.abs(_fp(P))
    bar = 0.25 * tol * A.sum(axis=1).max()
    ext = []
    for off, sign in ((oy, -1), (oy, 1), (ox, -1), (ox, 1)):
        side = sign * off  # distance beyond the owner on this side (negative: the other side)
        e = 0
        while (A * (side > e)).sum(axis=1).max() > bar:
            e += 1
        ext.append(e)
    return tuple(ext)


def truncate_propagator(P: np.ndarray, window: Window, shape, ext) -> np.ndarray:
    """P with every entry outside the owner's box -ly <= oy <= hy, -lx <= ox <= hx zeroed."""
    ly, hy, lx, hx = ext
    oy, ox = window_offsets(window, shape)
    keep = (oy >= -ly) & (oy <= hy) & (ox >= -lx) & (ox <= hx)
    return np.where(keep, _fp(P), 0.0)


def porous_phi(u: np.ndarray, m: float) -> np.ndarray:
    """The porous-medium nonlinearity c^m of Eq. porous (Sec. 4.2), extended oddly,
    |u|^(m-1) u, so that it stays defined where a step undershoots below zero."""
    return np.abs(u) ** (m - 1.0) * u


def residual(Xg: sp.csr_matrix, u: np.ndarray, dt: float = 0.0, reaction: bool = False,
             porous_m: float = 0.0):
    """dt * F(u): X u (linear, g = 0) plus dt * (u - u^3) when the reaction is on.
    Porous medium (porous_m = m > 1): dt * F(u) = X phi(u) with phi(u) = |u|^(m-1) u, the
    second-difference operator applied to c^m (Eq. porous)."""
    if porous_m:
        return Xg @ porous_phi(u, porous_m)
    r = Xg @ u
    if reaction:
        r = r + dt * (u - u ** 3)
    return r


def jacobian(Xg: sp.csr_matrix, u: np.ndarray, dt: float, reaction: bool,
             porous_m: float = 0.0) -> sp.csr_matrix:
    """dt * F'(u) = X + dt * diag(1 - 3 u^2) (just X for a linear problem): the Jacobian of the
    exponential Euler-Rosenbrock step (Sec. 4).
    Porous medium: dt * F'(u) = X diag(phi'(u)), phi'(u) = m |u|^(m-1) (chain rule through
    the operator: column j of X scaled by phi'(u_j))."""
    if porous_m:
        return (Xg @ sp.diags(porous_m * np.abs(u) ** (porous_m - 1.0))).tocsr()
    if not reaction:
        return Xg
    return (Xg + sp.diags(dt * (1.0 - 3.0 * u ** 2))).tocsr()


def lem_step(Xg, u, windows, props, mode: str = "phi", dt: float = 0.0,
             reaction: bool = False, tiles=None, porous_m: float = 0.0):
    """One LEM step u^n -> u^{n+1} (Sec. 3, steps 1-3; all windows read u^n).

    phi: u_D <- u_D + P_i (dt F(u^n))|_{M_i}   (Eq. lem, neighbours frozen at t^n)
    exp: u_D <- P_i u^n|_{M_i}                   (zero data at the artificial boundary)
    Only the owner rows D_i are written (buffer values discarded). ``tiles`` limits the
    update to a subset of windows; other entries of the result keep u^n.
    """
    u = _fp(u)
    out = u.copy()
    sel = range(len(windows)) if tiles is None else tiles
    if mode == "phi":
        r = residual(Xg, u, dt, reaction, porous_m)
        for i in sel:
            w = windows[i]
            out[w.D] = u[w.D] + props[i] @ r[w.M]
    else:
        for i in sel:
            w = windows[i]
            out[w.D] = props[i] @ u[w.M]
    return out


def lem_run(Xg, u0, windows, nsteps: int, mode: str = "phi", dt: float = 0.0,
            reaction: bool = False, refresh: int = 0, porous_m: float = 0.0,
            trunc_tol=None, shape=None):
    """nsteps LEM steps. Linear problems build the propagators once (Sec. 4: phi matrices
    computed at the first step only). With the reaction (or the porous-medium nonlinearity),
    the Jacobian and its propagators are rebuilt from the current state every ``refresh``
    steps (0 = never after step 0): the exponential Euler-Rosenbrock step with a frozen
    Jacobian (Sec. 4). With ``trunc_tol`` (and the mesh ``shape``) every propagator is
    truncated to its box (``truncation_extents``) right after each build."""
    u = _fp(u0).copy()
    props = None
    nonlinear = reaction or porous_m
    for n in range(nsteps):
        if props is None or (nonlinear and refresh > 0 and n % refresh == 0):
            props = local_propagators(jacobian(Xg, u, dt, reaction, porous_m), windows, mode)
            if trunc_tol is not None:
                props = [truncate_propagator(P, w, shape, truncation_extents(P, w, shape, trunc_tol))
                         for P, w in zip(props, windows)]
        u = lem_step(Xg, u, windows, props, mode, dt, reaction, porous_m=porous_m)
    return u


def rb3_defect(u, U, um, dt: float):
    """dt (G(U) - G(u)) with G(v) = F(v) - J(u_m) v (the exprb32 defect; Sec. 4.2), the part of F(v) = A v + v - v^3 that the
    frozen Jacobian J(u_m) = A + diag(1 - 3 u_m^2) leaves out. The linear parts cancel, so
    the defect is pointwise: dt [(U - U^3) - (u - u^3) - (1 - 3 u_m^2)(U - u)]."""
    return dt * ((U - U ** 3) - (u - u ** 3) - (1.0 - 3.0 * um ** 2) * (U - u))


def lem_step_rb3(Xg, u, windows, props1, props3, dt: float, um):
    """exprb32 in LEM form, with X_m = dt J(u_m) (the Jacobian at the last refresh):
        U       = u + phi_1(X_m) dt F(u)               window by window, owner rows (Eq. lem)
        u^{n+1} = U + 2 phi_3(X_m) dt (G(U) - G(u))   window by window, owner rows
    Both stages read the whole previous stage (Jacobi, as in Sec. 3)."""
    u = _fp(u)
    U = lem_step(Xg, u, windows, props1, "phi", dt, True)
    d = rb3_defect(u, U, um, dt)
    out = U.copy()
    for i, w in enumerate(windows):
        out[w.D] = U[w.D] + 2.0 * (props3[i] @ d[w.M])
    return out


def lem_run_rb3(Xg, u0, windows, nsteps: int, dt: float, refresh: int = 0):
    """nsteps exprb32 LEM steps (Sec. 4.2's third-order exponential Rosenbrock method in the
    form of Eq. lem); the Jacobian (and both propagator sets) are rebuilt from the current
    state every ``refresh`` steps (0 = only at the first step)."""
    u = _fp(u0).copy()
    props1 = props3 = um = None
    for n in range(nsteps):
        if props1 is None or (refresh > 0 and n % refresh == 0):
            um = u.copy()
            J = jacobian(Xg, um, dt, True)
            props1 = local_propagators(J, windows, "phi")
            props3 = local_propagators(J, windows, "phi3")
        u = lem_step_rb3(Xg, u, windows, props1, props3, dt, um)
    return u


# --------------------------------------------------------------------------- global reference
def global_step(Xg, u, dt: float = 0.0, reaction: bool = False, J=None, porous_m: float = 0.0):
    """Global exponential-Euler step u + phi_1(J) dt F(u) with dense phi_1 (small N only).

    For a linear problem with g = 0 this is exp(X) u exactly (Sec. 2 identity).
    """
    Jm = jacobian(Xg, u, dt, reaction, porous_m) if J is None else J
    return u + phi1(Jm.toarray()) @ residual(Xg, u, dt, reaction, porous_m)


def global_run(Xg, u0, nsteps: int, dt: float = 0.0, reaction: bool = False, refresh: int = 0,
               porous_m: float = 0.0):
    """nsteps global steps: exp(X)^nsteps u0 for a linear problem (Sec. 2 identity), else the
    exponential Euler-Rosenbrock step with the Jacobian refreshed every ``refresh`` steps
    (Sec. 4)."""
    u = _fp(u0).copy()
    if not reaction and not porous_m:
        E = expm_pade13(Xg.toarray())
        for _ in range(nsteps):
            u = E @ u
        return u
    J = None
    for n in range(nsteps):
        if J is None or (refresh > 0 and n % refresh == 0):
            J = jacobian(Xg, u, dt, reaction, porous_m)
        u = global_step(Xg, u, dt, reaction, J=J, porous_m=porous_m)
    return u


def global_step_rb3(Xg, u, dt: float, um):
    """exprb32 on the whole mesh with dense phi_1 and phi_3 of dt J(u_m) (small N only): the
    global third-order exponential Rosenbrock step of Sec. 4.2 that the LEM form approximates."""
    Jd = jacobian(Xg, um, dt, True).toarray()
    U = u + phi1(Jd) @ residual(Xg, u, dt, True)
    return U + 2.0 * (phik(Jd, 3) @ rb3_defect(u, U, um, dt))


def global_run_rb3(Xg, u0, nsteps: int, dt: float, refresh: int = 0):
    """nsteps global exprb32 steps (Sec. 4.2), u_m refreshed every ``refresh`` steps."""
    u = _fp(u0).copy()
    um = None
    for n in range(nsteps):
        if um is None or (refresh > 0 and n % refresh == 0):
            um = u.copy()
        u = global_step_rb3(Xg, u, dt, um)
    return u


def heat1d_eigenvalues(n: int, mu: float) -> np.ndarray:
    """Eigenvalues lambda_k = -4 mu sin^2(pi k / (2(n+1))), k = 1..n, of
    mu * tridiag(1, -2, 1) with homogeneous Dirichlet walls (eigenvectors sin(pi j k/(n+1))):
    the closed form of the global step (Sec. 2) for the 1D heat equation."""
    k = np.arange(1, n + 1)
    return -4.0 * mu * np.sin(np.pi * k / (2.0 * (n + 1))) ** 2


def heat1d_dst_modes(n: int, mu: float, amps: dict, nsteps: int) -> np.ndarray:
    """Exact global solution after ``nsteps`` steps (Sec. 2 identity) for
    u0 = sum_k a_k sin(pi k j/(n+1)), j = 1..n: every sine mode decays by exp(lambda_k) per step."""
    lam = heat1d_eigenvalues(n, mu)
    j = np.arange(1, n + 1)
    u = np.zeros(n)
    for k, a in amps.items():
        u += a * np.exp(nsteps * lam[k - 1]) * np.sin(np.pi * k * j / (n + 1))
    return u


def periodic2d_symbol(shape, coef) -> np.ndarray:
    """Fourier symbol of a constant dt-scaled 5-point stencil (Eq. spacedisc) on a periodic mesh:
    lambda(tx, ty) = C + W e^{-i tx} + E e^{i tx} + S e^{-i ty} + N e^{i ty}."""
    ny, nx = shape
    tx = 2 * np.pi * np.fft.fftfreq(nx)[None, :]
    ty = 2 * np.pi * np.fft.fftfreq(ny)[:, None]
    return (coef["C"] + coef["W"] * np.exp(-1j * tx) + coef["E"] * np.exp(1j * tx)
            + coef["S"] * np.exp(-1j * ty) + coef["N"] * np.exp(1j * ty))


def periodic2d_fft_step(u2d: np.ndarray, coef_dt: dict, nsteps: int = 1) -> np.ndarray:
    """Exact global step(s) exp(nsteps X) u (Sec. 2) for a constant-coefficient periodic 2D
    stencil (X is circulant, so the 2D DFT diagonalises it)."""
    lam = periodic2d_symbol(u2d.shape, coef_dt)
    return np.real(np.fft.ifft2(np.fft.fft2(u2d) * np.exp(nsteps * lam)))


def barenblatt1d(x: np.ndarray, t: float, m: float, A: float) -> np.ndarray:
    """The closed-form solution of Eq. porous in 1D quoted in Sec. 4.2 (Barenblatt):
    u(x, t) = t^-k (A^2 - k (m - 1) x^2 / (2 m t^(2k)))_+^(1/(m-1)) with k = 1/(m+1); the
    paper's t + t0 is the argument t here."""
    k = 1.0 / (m + 1.0)
    core = A * A - k * (m - 1.0) * x * x / (2.0 * m * t ** (2.0 * k))
    return t ** (-k) * np.maximum(core, 0.0) ** (1.0 / (m - 1.0))


def rel_l2(a, b) -> float:
    """||a - b||_2 / ||b||_2: the relative error the paper reports (Sec. 4), in the L2 norm."""
    a = _fp(a).ravel()
    b = _fp(b).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))
