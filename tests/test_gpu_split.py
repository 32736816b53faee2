"""GPU parity of the split-precision tensor-core LEM path (FP16 pieces of the propagator and
the residual, tcgen05 MMA with FP32 accumulation, float-float state) against the FP64 oracle.
Two tiers: "split" (three pieces per operand, six products) and "split_fast" (two pieces,
four products).

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


@pytest.mark.parametrize("prec", ["split", "split_fast"])
def test_split_is_eligible_and_uses_tensor_path(case512, prec):
    wl, _ = case512
    ctx = L.Lem.from_workload(wl, prec=prec)
    assert ctx.info()["split_path"] == 1


@pytest.mark.parametrize("prec", ["split", "split_fast"])
@pytest.mark.parametrize("steps", [1, 10, 100])
def test_split_512_vs_oracle(case512, steps, prec):
    wl, ref = case512
    ctx = L.Lem.from_workload(wl, prec=prec)
    u = torch.tensor(wl["u0"], device="cuda")
    ctx.step(u, steps)
    ctx.sync()
    err = rel_l2(u.cpu().numpy(), ref[steps])
    print(f"{prec} 512^2 {steps} steps rel_l2 = {err:.3e}")
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


def test_split_without_shared_propagator_paths():
    """1D heat has three propagator classes: LEM_PREC_SPLIT_FAST applies FP32 propagators
    with a float-float GEMV there (100 steps within the split bar of the oracle), and
    LEM_PREC_SPLIT falls back to the FP64 path."""
    wl = W.heat1d()
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    assert L.APPLY_PATHS[L.Lem.from_workload(wl, prec="split").info()["apply_path"]].startswith("fp64")
    ctx = L.Lem.from_workload(wl, prec="split_fast")
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


@pytest.mark.parametrize("side,tile,H", [
    (128, 8, 4),    # 16-wide windows, 64-row propagator (one M block, half masked)
    (128, 8, 7),    # 22-wide windows: K slice not a multiple of 16
    (96, 16, 5),    # 26-wide windows, 256 rows
    (160, 16, 8),   # 32-wide windows, ragged 10-tile grid
    (128, 32, 4),   # 40-wide windows, 1024 rows
])
def test_split_small_tiles_vs_oracle(side, tile, H):
    """Tile and overlap shapes of uneven-size batches (tile 8/16/32, H 4-8): window widths
    that are not multiples of the 16-wide MMA K step and propagators with fewer rows than an
    MMA block still take the tensor path and stay within the split bar."""
    wl = W.advdiff2d(side=side, tile=tile, overlap=H, nu=7.0, a=(2.0, 1.0), dt=2.0, ell=8.0, seed=11)
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    P = local_propagators(X, wins, "phi", tiles=[0])[0]
    props = [P] * len(wins)
    ref = wl["u0"].copy()
    for _ in range(20):
        ref = lem_step(X, ref, wins, props, "phi")
    ctx = L.Lem.from_workload(wl, prec="split")
    assert ctx.info()["split_path"] == 1
    u = torch.tensor(wl["u0"], device="cuda")
    ctx.step(u, 20)
    ctx.sync()
    err = rel_l2(u.cpu().numpy(), ref)
    print(f"split {side}^2 tile {tile} H {H} 20 steps rel_l2 = {err:.3e}")
    assert err <= TOL_SPLIT_100


def test_split_rough_decaying_field_100_steps():
    """A rough field (correlation length 8 h on a 64^2 mesh) under strong diffusion
    (nu dt / h^2 = 42) loses three orders of magnitude in 100 steps, so early rounding
    errors in its slow modes count against a much smaller final state. The three-piece tier
    keeps 100 steps within the bar; the two-piece tier is only reported."""
    p = W.batch_problems(n=20, seed=5, side_max=128)[4]
    assert p["shape"] == (64, 64) and p["tile"] == (32, 32) and p["overlap"] == (7, 7)
    X = assemble_operator(p["shape"], p["bc"], p["coef"], p["dt"])
    wins = decompose(p["shape"], p["bc"], p["tile"], p["overlap"])
    from oracle import lem_run
    ref = lem_run(X, p["u0"], wins, 100)
    errs = {}
    for prec in ("split", "split_fast"):
        ctx = L.Lem.from_workload(p, prec=prec)
        assert ctx.info()["split_path"] == 1
        u = torch.tensor(p["u0"], device="cuda")
        ctx.step(u, 100)
        ctx.sync()
        errs[prec] = rel_l2(u.cpu().numpy(), ref)
    print(f"rough decaying 64^2, 100 steps: rel_l2 {errs}")
    assert errs["split"] <= TOL_SPLIT_100


@pytest.mark.parametrize("prec", ["split", "split_fast"])
def test_step_host_pinned_pageable_and_device_agree_bit_for_bit(prec):
    """lem_step_host on a split context: with a pinned host buffer the conversion kernels read
    and write it in place, with a pageable one it is copied; both give the device step's bits."""
    wl = W.advdiff2d(side=256, ell=8.0, seed=31)
    dev, pin, pag = (L.Lem.from_workload(wl, prec=prec) for _ in range(3))
    u = torch.tensor(wl["u0"], device="cuda")
    dev.step(u, 6)
    dev.sync()
    pin.build()  # (the in-place path takes built contexts)
    assert L.APPLY_PATHS[pin.info()["apply_path"]] == "tc_split"
    hp = torch.tensor(wl["u0"]).pin_memory()
    pin.step_host(hp.numpy(), 6)
    hq = wl["u0"].copy()
    pag.step_host(hq, 6)
    ref = u.cpu().numpy()
    assert np.array_equal(hp.numpy(), ref)
    assert np.array_equal(hq, ref)


@pytest.mark.parametrize("prec", ["split", "split_fast"])
@pytest.mark.parametrize("nsteps", [1, 4])
@pytest.mark.parametrize("side,tile,H", [
    (160, 32, 8),              # 5 x 5 tiles; the padded 176-wide grid ends in a part tile
    (24, 8, 4),                # mesh smaller than one 64 x 32 residual tile: every halo wraps
    (96, 16, 5),               # 26-wide windows
    (128, (32, 16), (16, 8)),  # anisotropic windows (64 x 32)
])
def test_device_state_conversion_in_measuring_pass_matches_streaming_one(prec, nsteps, side, tile, H):
    """On a device state the measuring residual pass converts the FP64 state to float-float as
    it stages it (each mesh node written once); on a mapped pinned host state a separate
    streaming kernel converts it over the host link. Two calls in a row on each must give the
    same bits."""
    wl = W.advdiff2d(side=side, tile=tile, overlap=H, nu=7.0, a=(2.0, 1.0), dt=2.0, ell=8.0, seed=13)
    dev, pin = (L.Lem.from_workload(wl, prec=prec) for _ in range(2))
    assert dev.info()["split_path"] == 1
    pin.build()
    u = torch.tensor(wl["u0"], device="cuda")
    hp = torch.tensor(wl["u0"]).pin_memory()
    for _ in range(2):
        dev.step(u, nsteps)
        pin.step_host(hp.numpy(), nsteps)
        dev.sync()
        assert np.array_equal(hp.numpy(), u.cpu().numpy())
    assert not np.array_equal(hp.numpy(), wl["u0"])


def test_balanced_last_wave_matches_whole_units(monkeypatch):
    """1792^2 (tiles 32, 224 units of 128 owner rows x 128 windows on a 152-SM GB300): the
    full wave runs whole units and the remaining 72 units' window rows are spread over every
    CTA, a split unit finished by the CTA holding its first rows. The result must agree with
    whole units (LEM_SPLIT_BALANCE=0) up to the order of the correction sums, and both with
    the FP64 GPU LEM within the split tier's bar."""
    wl = W.advdiff2d(side=1792, seed=7)
    steps = 30
    monkeypatch.setenv("LEM_SPLIT_BALANCE", "0")
    whole = L.Lem.from_workload(wl, prec="split")
    monkeypatch.delenv("LEM_SPLIT_BALANCE")
    bal = L.Lem.from_workload(wl, prec="split")
    fp64 = L.Lem.from_workload(wl, prec="fp64")
    u_b = torch.tensor(wl["u0"], device="cuda")
    u_w = torch.tensor(wl["u0"], device="cuda")
    u_d = torch.tensor(wl["u0"], device="cuda")
    bal.step(u_b, steps)
    whole.step(u_w, steps)
    fp64.step(u_d, steps)
    torch.cuda.synchronize()
    b, w, d = (x.cpu().numpy() for x in (u_b, u_w, u_d))
    assert rel_l2(b, w) <= 1e-8
    assert rel_l2(b, d) <= TOL_SPLIT_100 and rel_l2(w, d) <= TOL_SPLIT_100
