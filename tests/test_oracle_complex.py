"""Pins for the oracle on complex problems: the 1D Schroedinger test of Sec. 4.1
(c_t = (i/2) c_xx - i (kappa/2) x^2 c, periodic, centred differences).

Independent checks: complex scalar exp and phi_1 closed forms; the free equation (kappa = 0)
against its Fourier closed form; unitarity of the global step (A = i H with H real symmetric);
one window covering the mesh equals the global step; the LEM error shrinks with the buffer;
the rows of the paper's Schroedinger table (LEM adds nothing to the error at its buffers; the
error against a pseudospectral reference does not depend on the time step).
"""
import os

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import assemble_operator, decompose, expm_pade13, global_run, lem_run, phi1, rel_l2
from paper_1505_02248_gb300 import workloads as W


@pytest.mark.parametrize("z", [0.3j, -2.0 + 5.0j, 12.0j, -0.001 + 0.0j, 1.5 - 0.7j])
def test_complex_scalar_exp_phi1(z):
    e = expm_pade13(np.array([[z]]))[0, 0]
    assert abs(e - np.exp(z)) <= 1e-14 * max(1.0, abs(np.exp(z)))
    if abs(z) < 0.1:  # the series: (e^z - 1) / z cancels here
        ref, t = 0.0, 1.0
        for k in range(1, 25):
            t *= z / (k + 1) if k > 1 else 0.5 * z
            ref += t
        ref += 1.0
    else:
        ref = (np.exp(z) - 1.0) / z
    assert abs(phi1(np.array([[z]]))[0, 0] - ref) <= 1e-14 * max(1.0, abs(ref))


def test_free_schroedinger_fourier_closed_form():
    wl = W.schrodinger1d(n=128, kappa=0.0, mu=2.0)
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    steps = 7
    got = global_run(X, wl["u0"], steps)
    k = np.arange(128)
    lam = 1j / 2 * (-4.0 * np.sin(np.pi * k / 128) ** 2 / wl["h"] ** 2) * wl["dt"]
    ref = np.fft.ifft(np.fft.fft(wl["u0"]) * np.exp(steps * lam))
    assert rel_l2(got, ref) <= 1e-12


def test_global_step_is_unitary():
    wl = W.schrodinger1d(n=160, mu=2.0)
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    Xd = X.toarray()
    assert np.abs(Xd + Xd.conj().T).max() <= 1e-12 * np.abs(Xd).max()   # anti-Hermitian
    u = global_run(X, wl["u0"], 20)
    assert abs(np.linalg.norm(u) / np.linalg.norm(wl["u0"]) - 1.0) <= 1e-12


def test_complex_lem_one_window_is_global_and_buffer_helps():
    wl = W.schrodinger1d(n=160, mu=2.0, tile=40)
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    g = global_run(X, wl["u0"], 10)
    one = decompose(wl["shape"], wl["bc"], (160,), (0,))
    assert rel_l2(lem_run(X, wl["u0"], one, 10), g) <= 1e-13
    e = [rel_l2(lem_run(X, wl["u0"], decompose(wl["shape"], wl["bc"], (40,), (B,)), 10), g) for B in (5, 10, 20)]
    assert e[0] > e[1] > e[2] and e[2] < 1e-6


def _table2():
    rows, kv = [], {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_table2_schroedinger.txt")) as f:
        for line in f:
            parts = line.split()
            if not parts or line.startswith("#"):
                continue
            if parts[0][0].isdigit():
                rows.append((float(parts[0]), int(parts[1])))
            else:
                kv[parts[0]] = [float(v) for v in parts[1:]]
    return rows, kv


def test_paper_table2_rows():
    """Every (mu, B, D) of the Schroedinger table (Sec. 4.1): the LEM solution at T = 1 stays
    within 1 % of the paper's error level of the global exponential step, so the table's uniform
    error is the discretisation's, not the decomposition's. For a linear autonomous problem the
    exponential step is exact in time (Sec. 2), so the global error against the semi-discrete
    pseudospectral solution is the same at both time steps."""
    rows, kv = _table2()
    assert len(rows) == 2 and kv["subdomains"] == [1, 2, 4, 5, 10]
    T, level = kv["T"][0], kv["rel_error"][0]
    n, L, kappa = int(kv["npoints"][0]), kv["L"][0], kv["kappa"][0]
    glob_err = []
    for mu, B in rows:
        wl = W.schrodinger1d(n=n, L=L, kappa=kappa, mu=mu)
        X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
        steps = int(round(T / wl["dt"]))
        assert abs(steps * wl["dt"] - T) < 1e-12
        g = global_run(X, wl["u0"], steps)
        for D in kv["subdomains"]:
            wins = decompose(wl["shape"], wl["bc"], (n // int(D),), (B,))
            assert rel_l2(lem_run(X, wl["u0"], wins, steps), g) <= 1e-2 * level
        # pseudospectral reference: the same equation with Fourier differentiation, exact in time
        k = 2 * np.pi * np.fft.fftfreq(n, d=wl["h"])
        D2 = np.fft.ifft(-(k ** 2)[:, None] * np.fft.fft(np.eye(n), axis=0), axis=0)
        A = 0.5j * D2 - 0.5j * kappa * np.diag(wl["x"] ** 2)
        glob_err.append(rel_l2(g, sl.expm(T * A) @ wl["u0"]))
    assert abs(glob_err[0] - glob_err[1]) <= 1e-9 * glob_err[0]
