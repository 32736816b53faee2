"""Pins for the oracle's matrix functions: Pade-13 scaling-and-squaring exp and phi_1.

Each test checks the oracle against something other than itself: published coefficients,
closed forms, an independent library (scipy), arbitrary precision (mpmath) or identities
that a dropped term, a wrong sign or a transposed operand would break.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import THETA13, expm_pade13, pade13_coefficients, phi1, squaring_count

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _ints(name):
    with open(os.path.join(GOLD, name)) as f:
        return [int(x) for x in f.read().split("\n") if x.strip() and not x.startswith("#")]


def test_pade13_coefficients_match_published_integers():
    ints = _ints("pade13_numerator_integers.txt")
    b = pade13_coefficients()
    assert len(b) == 14 == len(ints)
    for j in range(14):
        assert b[j] == pytest.approx(ints[j] / ints[0], rel=1e-15)


def test_pade13_scalar_accuracy_up_to_theta():
    # r_13(x) = p(x)/p(-x) evaluated in 50-digit arithmetic: for |x| <= theta_13 it meets
    # e^x to about unit roundoff times |x| (Higham's backward-error design).
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    b = [mpmath.mpf(v) for v in _ints("pade13_numerator_integers.txt")]  # exact integers
    for x in np.linspace(-THETA13, THETA13, 41):
        xm = mpmath.mpf(float(x))
        p = sum(bj * xm ** j for j, bj in enumerate(b))
        q = sum(bj * (-xm) ** j for j, bj in enumerate(b))
        rel = abs(p / q - mpmath.exp(xm)) / mpmath.exp(xm)
        assert rel <= 2.3e-16 * max(1.0, abs(x))


@pytest.mark.parametrize("norm,s", [(0.0, 0), (1.0, 0), (THETA13, 0), (THETA13 * 1.0000001, 1),
                                    (2 * THETA13, 1), (2 * THETA13 * 1.0000001, 2),
                                    (40.0, 3), (172.0, 6), (1e6, 18)])
def test_squaring_count(norm, s):
    assert squaring_count(norm) == s


def test_expm_zero_is_identity():
    for n in (1, 4, 17):
        assert np.array_equal(expm_pade13(np.zeros((n, n))), np.eye(n))


def test_expm_diagonal():
    d = np.array([-300.0, -40.0, -1.0, 0.0, 0.5, 3.0])
    E = expm_pade13(np.diag(d))
    assert np.allclose(np.diag(E), np.exp(d), rtol=1e-13, atol=1e-300)
    assert np.abs(E - np.diag(np.diag(E))).max() == 0.0


def test_expm_nilpotent_jordan_block_exact_series():
    n, t = 8, 3.7
    J = t * np.eye(n, k=1)
    exact = sum(np.linalg.matrix_power(J, k) / math.factorial(k) for k in range(n))
    assert np.allclose(expm_pade13(J), exact, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("theta", [0.3, 5.0, 40.0])
def test_expm_rotation_closed_form(theta):
    X = np.array([[0.0, theta], [-theta, 0.0]])
    R = np.array([[math.cos(theta), math.sin(theta)], [-math.sin(theta), math.cos(theta)]])
    assert np.allclose(expm_pade13(X), R, atol=1e-12 * max(1, theta))


def test_expm_transposition():
    X = np.random.default_rng(5).standard_normal((9, 9))
    assert np.allclose(expm_pade13(X.T), expm_pade13(X).T, rtol=1e-13, atol=1e-14)


def test_expm_symmetric_vs_eigendecomposition():
    rng = np.random.default_rng(1)
    G = rng.standard_normal((40, 40))
    S = -(G @ G.T) / 2.0  # symmetric negative semi-definite, norm ~ 60
    lam, V = np.linalg.eigh(S)
    ref = (V * np.exp(lam)) @ V.T
    assert np.abs(expm_pade13(S) - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("scale", [0.1, 3.0, 30.0, 200.0])
def test_expm_vs_scipy(scale):
    rng = np.random.default_rng(int(scale * 10))
    X = scale * rng.standard_normal((24, 24)) / math.sqrt(24)
    X -= 1.5 * scale * np.eye(24)  # stable spectrum, non-normal
    ref = sl.expm(X)
    assert np.abs(expm_pade13(X) - ref).max() <= 1e-11 * np.abs(ref).max()


def test_expm_vs_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(7)
    for n, scale in ((3, 2.0), (6, 12.0), (10, 30.0)):
        X = scale * rng.standard_normal((n, n)) / math.sqrt(n)
        ref = np.array(mpmath.expm(mpmath.matrix(X.tolist())).tolist(), dtype=float)
        assert np.abs(expm_pade13(X) - ref).max() <= 1e-12 * np.abs(ref).max()


def test_expm_semigroup():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((30, 30)) - 3 * np.eye(30)
    E1 = expm_pade13(X)
    assert np.allclose(E1 @ E1, expm_pade13(2 * X), rtol=1e-11, atol=1e-14)
    assert np.allclose(E1 @ expm_pade13(-X), np.eye(30), atol=1e-11)


@pytest.mark.parametrize("z", [-700.0, -60.0, -3.0, -1e-8, 0.0, 1e-8, 0.7, 4.0])
def test_phi1_scalar_closed_form(z):
    ref = 1.0 if z == 0.0 else math.expm1(z) / z
    assert phi1(np.array([[z]]))[0, 0] == pytest.approx(ref, rel=1e-13)


def test_phi1_matrix_identities():
    rng = np.random.default_rng(11)
    X = 4.0 * rng.standard_normal((20, 20)) / math.sqrt(20) - 2.0 * np.eye(20)
    P = phi1(X)
    E = sl.expm(X)
    assert np.allclose(np.eye(20) + X @ P, E, rtol=1e-12, atol=1e-13)
    assert np.allclose(P, np.linalg.solve(X, E - np.eye(20)), rtol=1e-10, atol=1e-12)
    assert np.allclose(X @ P, P @ X, atol=1e-12)  # phi_1(X) commutes with X
    assert np.array_equal(phi1(np.zeros((5, 5))), np.eye(5))


def test_phi1_series_small_norm():
    rng = np.random.default_rng(13)
    X = 0.3 * rng.standard_normal((8, 8))
    S = np.zeros((8, 8))
    T = np.eye(8)
    for k in range(30):
        S += T / math.factorial(k + 1)
        T = T @ X
    assert np.allclose(phi1(X), S, rtol=1e-14, atol=1e-15)
