"""Per-tile propagators (variable coefficients, the u - u^3 reaction with Jacobian refresh):
the batched GEMV apply against the oracle. Every tile has its own local operator, so every
tile gets its own Pade-13 phi_1 propagator (Sec. 3, Sec. 4 exponential Euler-Rosenbrock)."""
import numpy as np
import pytest

from oracle import (assemble_operator, decompose, jacobian, lem_run, lem_step, local_propagators, rel_l2)
from paper_1505_02248_gb300 import lem as L
from paper_1505_02248_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_02248_gb300 import build as B
    B.build()
    L.load()


def _run(wl, prec, steps):
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    ref = lem_run(X, wl["u0"], wins, steps, "phi", wl["dt"], wl["reaction"], wl.get("refresh", 0))
    ctx = L.Lem.from_workload(wl, prec=prec)
    u = torch.tensor(wl["u0"], device="cuda")
    ctx.step(u, steps)
    ctx.sync()
    path = L.APPLY_PATHS[ctx.info()["apply_path"]]
    ctx.close()
    return rel_l2(u.cpu().numpy(), ref), path


def test_fp64_gemv_reaction_refresh():
    wl = W.vardiff2d(side=96, tile=16, overlap=6)
    wl["refresh"] = 2
    err, path = _run(wl, "fp64", 6)
    assert path == "fp64_gemv" and err <= 1e-12


def test_fp64_gemv_dirichlet_no_reaction():
    wl = W.vardiff2d(side=128, tile=16, overlap=6)
    wl["reaction"] = False
    err, path = _run(wl, "fp64", 5)
    assert path == "fp64_gemv" and err <= 1e-12


def test_f32_gemv_reaction_within_split_bar():
    wl = W.vardiff2d(side=96, tile=16, overlap=6)
    wl["refresh"] = 5
    err, path = _run(wl, "split_fast", 20)
    print(f"f32 gemv vardiff 96^2 20 steps rel_l2 = {err:.3e}")
    assert path == "f32_gemv" and err <= 1e-6


def test_vardiff_512_sampled_tiles():
    """512^2 (1024 tiles of 16^2 + H 6, 784-node windows): one FP64 step on sampled tiles,
    each with its own propagator built from the Jacobian at u0."""
    wl = W.vardiff2d(side=512, tile=16, overlap=6)
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    ctx = L.Lem.from_workload(wl, prec="fp64")
    u = torch.tensor(wl["u0"], device="cuda")
    ctx.step(u, 1)
    ctx.sync()
    got = u.cpu().numpy()
    sample = [0, 31, 500, 1023]
    Xj = jacobian(X, wl["u0"], wl["dt"], True)
    props = local_propagators(Xj, wins, "phi", tiles=sample)
    ref = lem_step(X, wl["u0"], wins, props, "phi", wl["dt"], True, tiles=sample)
    for t in sample:
        D = wins[t].D
        assert rel_l2(got[D], ref[D]) <= 1e-12
