"""GPU parity of the split-precision tensor-core LEM path (FP16 hi/lo propagator and
residual, tcgen05 MMA with FP32 accumulation, float-float state) against the FP64 oracle.

Bar (stated for the mixed-precision path): within 1e-6 relative L2 of the FP64 oracle LEM
after 100 steps. At 2048^2 the 100-step reference is the FP64 GPU path, itself pinned to the
oracle within 1e-12 (tests/test_gpu_fp64.py), plus a direct oracle check on sampled tiles."""
import os

import numpy as np
import pytest

from oracle import assemble_operator, decompose, lem_step, local_propagators, rel_l2
from paper_1505_02248_gb300 import lem as L
from paper_1505_02248_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_SPLIT_100 = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_02248_gb300 import build as B
    B.build()
    L.load()


@pytest.fixture(scope="module")
def case512():
    wl = W.advdiff2d(side=512)
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    P = local_propagators(X, wins, "phi", tiles=[0])[0]
    props = [P] * len(wins)
    ref = {0: wl["u0"].copy()}
    u = wl["u0"].copy()
    for n in range(1, 101):
        u = lem_step(X, u, wins, props, "phi")
        if n in (1, 10, 100):
            ref[n] = u.copy()
    return wl, ref


def test_split_is_eligible_and_uses_tensor_path(case512):
    wl, _ = case512
    ctx = L.Lem.from_workload(wl, prec="split")
    assert ctx.info()["split_path"] == 1


@pytest.mark.parametrize("steps", [1, 10, 100])
def test_split_512_vs_oracle(case512, steps):
    wl, ref = case512
    ctx = L.Lem.from_workload(wl, prec="split")
    u = torch.tensor(wl["u0"], device="cuda")
    ctx.step(u, steps)
    ctx.sync()
    err = rel_l2(u.cpu().numpy(), ref[steps])
    print(f"split 512^2 {steps} steps rel_l2 = {err:.3e}")
    assert err <= TOL_SPLIT_100


def test_split_steps_compose(case512):
    """Ten calls of 10 steps equal one call of 100 steps within the same bar."""
    wl, ref = case512
    ctx = L.Lem.from_workload(wl, prec="split")
    u = torch.tensor(wl["u0"], device="cuda")
    for _ in range(10):
        ctx.step(u, 10)
    ctx.sync()
    assert rel_l2(u.cpu().numpy(), ref[100]) <= TOL_SPLIT_100


def test_split_full_size_100_steps():
    wl = W.advdiff2d()
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    split = L.Lem.from_workload(wl, prec="split")
    fp64 = L.Lem.from_workload(wl, prec="fp64")
    u_s = torch.tensor(wl["u0"], device="cuda")
    u_d = torch.tensor(wl["u0"], device="cuda")
    # one step against the oracle on sampled tiles
    split.step(u_s, 1)
    split.sync()
    P = local_propagators(X, wins, "phi", tiles=[0])[0]
    sample = [0, 63, 4032, 4095, 2080, 777]
    props = [P if i in sample else None for i in range(len(wins))]
    ref1 = lem_step(X, wl["u0"], wins, props, "phi", tiles=sample)
    got = u_s.cpu().numpy()
    # one step carries the FP16-slice representation error of P and r (about 2^-22 of each
    # row / column maximum, times the cancellation in the window sums); it does not compound
    for t in sample:
        D = wins[t].D
        assert rel_l2(got[D], ref1[D]) <= 5e-7
    # 100 steps against the FP64 path
    split.step(u_s, 99)
    fp64.step(u_d, 100)
    torch.cuda.synchronize()
    err = rel_l2(u_s.cpu().numpy(), u_d.cpu().numpy())
    print(f"split 2048^2 100 steps rel_l2 vs fp64 = {err:.3e}")
    assert err <= TOL_SPLIT_100


def test_split_without_shared_propagator_uses_f32_gemv():
    """1D heat has three propagator classes: LEM_PREC_SPLIT applies FP32 propagators with a
    float-float GEMV there; 100 steps stay within the split bar of the oracle."""
    wl = W.heat1d()
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    ctx = L.Lem.from_workload(wl, prec="split")
    assert L.APPLY_PATHS[ctx.info()["apply_path"]] == "f32_gemv"
    u = torch.tensor(wl["u0"], device="cuda")
    ctx.step(u, 100)
    ctx.sync()
    from oracle import lem_run
    assert rel_l2(u.cpu().numpy(), lem_run(X, wl["u0"], wins, 100)) <= TOL_SPLIT_100


@pytest.fixture(scope="module")
def shared_P():
    """The 1024 x 2304 phi_1 propagator shared by every tile of the tile-32 / H-8 workloads."""
    wl = W.advdiff2d(side=128)
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    return local_propagators(X, wins, "phi", tiles=[0])[0]


@pytest.mark.parametrize("side", [160, 384, 448])
def test_split_ragged_tile_grids_vs_oracle(shared_P, side):
    """Tile grids that do not fill whole 128/256-window blocks (5, 12, 14 tiles per side):
    the overhanging windows are zero-filled by TMA and skipped by the epilogue."""
    wl = W.advdiff2d(side=side, ell=8.0)
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    props = [shared_P] * len(wins)
    ref = wl["u0"].copy()
    for _ in range(10):
        ref = lem_step(X, ref, wins, props, "phi")
    ctx = L.Lem.from_workload(wl, prec="split")
    assert ctx.info()["split_path"] == 1
    u = torch.tensor(wl["u0"], device="cuda")
    ctx.step(u, 10)
    ctx.sync()
    assert rel_l2(u.cpu().numpy(), ref) <= TOL_SPLIT_100
