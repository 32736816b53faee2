"""The porous-medium problem (Sec. 4.2, Eq. porous: c_t = (c^m)_xx, m = 3) through the C-ABI
against the oracle. The Jacobian X diag(phi'(u)) depends on the state, so every tile has its
own propagator, rebuilt from the current state every `refresh` steps (exponential
Euler-Rosenbrock, Sec. 4). 1D at the paper's size (400 cells, Barenblatt datum) and a 2D case
whose windows wrap on a periodic axis.

Bars: FP64 within 1e-12 relative L2; the split tiers (tensor-core built propagators, FP32
propagators for split_fast) within their 1e-6 bar."""
import numpy as np
import pytest

from oracle import assemble_operator, barenblatt1d, decompose, lem_run, rel_l2
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
    ref = lem_run(X, wl["u0"], wins, steps, "phi", wl["dt"], False, wl["refresh"], porous_m=wl["porous_m"])
    ctx = L.Lem.from_workload(wl, prec=prec)
    u = torch.tensor(wl["u0"], device="cuda")
    ctx.step(u, steps)
    ctx.sync()
    path = L.APPLY_PATHS[ctx.info()["apply_path"]]
    ctx.close()
    got = u.cpu().numpy()
    return got, rel_l2(got, ref), path


@pytest.mark.parametrize("refresh", [1, 5])
@pytest.mark.parametrize("prec,bar,want", [("fp64", 1e-12, "fp64_gemv"), ("split", 1e-6, "fp64_gemv"),
                                           ("split_fast", 1e-6, "f32_gemv")])
def test_porous1d_barenblatt_vs_oracle(prec, bar, want, refresh):
    wl = W.porous1d(n=400, refresh=refresh)
    steps = 40
    got, err, path = _run(wl, prec, steps)
    print(f"porous1d 400 {prec} refresh {refresh}: {steps} steps rel_l2 {err:.2e}")
    assert path == want and err <= bar
    # still the Barenblatt solution (the oracle is 7.5e-4 from it here); the mass drifts only by
    # the decomposition error (not an LEM invariant: 3.5e-10 in the oracle)
    ref = barenblatt1d(wl["x"], wl["t0"] + steps * wl["dt"], wl["porous_m"], wl["A"])
    assert rel_l2(got, ref) <= 1e-2
    assert abs(got.sum() / wl["u0"].sum() - 1.0) <= (1e-8 if prec != "split_fast" else 1e-5)


def _porous2d():
    ny, nx = 40, 48
    h = 0.1
    yy, xx = np.meshgrid((np.arange(ny) - ny / 2 + 0.5) * h, (np.arange(nx) - nx / 2 + 0.5) * h, indexing="ij")
    u0 = np.sqrt(np.maximum(1.0 - (xx * xx + yy * yy) / 1.2 ** 2, 0.0)).ravel()
    c = 1.0 / h ** 2
    coef = {"C": -4.0 * c, "W": c, "E": c, "S": c, "N": c}
    # dt = h^2: stability parameter 3 on the largest diffusivity, phi'(max u0) = 3
    return dict(shape=(ny, nx), bc=("dirichlet", "periodic"), coef=coef, dt=h * h,
                tile=(8, 16), overlap=(4, 6), u0=u0, reaction=False, porous_m=3.0, refresh=2)


@pytest.mark.parametrize("prec,bar", [("fp64", 1e-12), ("split_fast", 1e-6)])
def test_porous2d_vs_oracle(prec, bar):
    wl = _porous2d()
    _, err, _ = _run(wl, prec, 6)
    print(f"porous2d 40x48 {prec}: 6 steps rel_l2 {err:.2e}")
    assert err <= bar


def test_porous_refused_by_batches_and_the_allocation_free_step():
    wl = W.porous1d(n=400, refresh=0)
    ctx = L.Lem.from_workload(wl)
    u = torch.tensor(wl["u0"], device="cuda")
    ctx.step(u, 1)
    with pytest.raises(L.LemError):
        ctx.step_noalloc(u, 1)
    with pytest.raises(L.LemError):
        L.Batch([ctx], [u])
    ctx.close()
