"""Pins for the oracle on complex problems: the 1D Schroedinger test of Sec. 4.1
(c_t = (i/2) c_xx - i (kappa/2) x^2 c, periodic, centred differences).

Independent checks: complex scalar exp and phi_1 closed forms; the free equation (kappa = 0)
against its Fourier closed form; unitarity of the global step (A = i H with H real symmetric);
one window covering the mesh equals the global step; the LEM error shrinks with the buffer.
"""
import numpy as np
import pytest

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
