"""Truncated propagators on the GPU (Sec. 2, Theorem 1: off-band decay of the local
exponentials) against the oracle's truncated LEM.

The library picks each class's box from the tolerance on the GPU (lem_set_truncation); the
extents must equal the oracle's, side by side, for every class, and the truncated steps must
match the oracle's truncated LEM: FP64 boxes within 1e-12 relative L2, FP32 boxes (split_fast)
within 1e-6. Cases: 1D periodic upwind advection-diffusion (asymmetric box), 1D Dirichlet
heat with clipped wall windows and a ragged last tile (several classes), EXP mode, 2D
periodic advection-diffusion, and 2D variable coefficients with the reaction and Jacobian
refreshes (a box per tile, recomputed after every rebuild)."""
import numpy as np
import pytest

from oracle import (assemble_operator, decompose, jacobian, lem_run, local_propagators, rel_l2,
                    truncation_extents)
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


def _adv1d(n=512, mu=2.0, c=1.0, tile=64, H=16, bc="periodic"):
    coef = W.stencil_advdiff_1d(mu, c, 1.0, upwind=True)
    return dict(shape=(n,), bc=(bc,), coef=coef, dt=1.0, tile=(tile,), overlap=(H,),
                u0=W.grf_1d(n, 6.0, 5), reaction=False)


def _check_extents(ctx, wl, tol, props_fn):
    """Every class's GPU machine equals the oracle's for a tile of that class."""
    wins = decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    seen = {}
    for t in range(len(wins)):
        seen.setdefault(ctx.tile_class(t), t)
    kept = 0
    for c, t in seen.items():
        P = props_fn(wins, t)
        want = truncation_extents(P, wins[t], wl["shape"], tol)
        got, nv = ctx.band(c)
        assert got == want, f"class {c} (tile {t}): GPU box {got}, oracle {want}"
        kept += nv
    return seen, kept


CASES = {
    "adv1d_periodic": (lambda: _adv1d(), 1e-8, "phi"),
    "heat1d_dirichlet_ragged": (lambda: W.heat1d(n=1000, tile=64, overlap=16, mu=3.0), 1e-10, "phi"),
    "heat1d_exp": (lambda: W.heat1d(n=512, tile=64, overlap=16, mu=2.0), 1e-10, "exp"),
    "advdiff2d_periodic": (lambda: W.advdiff2d(side=64, tile=16, overlap=8, nu=1.0, a=(1.0, 0.5), dt=1.0,
                                               ell=4.0), 1e-8, "phi"),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "split_fast"])
def test_truncated_steps_vs_oracle(case, prec):
    make, tol, mode = CASES[case]
    wl = make()
    steps = 20
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    ref = lem_run(X, wl["u0"], wins, steps, mode, trunc_tol=tol, shape=wl["shape"])
    full = lem_run(X, wl["u0"], wins, steps, mode)
    ctx = L.Lem.from_workload(wl, prec=prec, mode=mode)
    ctx.set_truncation(tol)
    fp32 = prec == "split_fast" and mode == "phi"
    assert L.APPLY_PATHS[ctx.info()["apply_path"]] == ("f32_band" if fp32 else "fp64_band")
    u = torch.tensor(wl["u0"], device="cuda")
    ctx.step(u, steps)
    ctx.sync()
    got = u.cpu().numpy()
    _, kept = _check_extents(ctx, wl, tol, lambda ws, t: local_propagators(X, ws, mode, tiles=[t])[t])
    info = ctx.info()
    ctx.close()
    err = rel_l2(got, ref)
    print(f"{case} {prec}: rel_l2 vs oracle truncated {err:.2e}; truncated vs full LEM "
          f"{rel_l2(ref, full):.2e}; {info['nclasses']} classes")
    assert err <= (1e-6 if fp32 else 1e-12)


def test_truncation_with_reaction_refresh_per_tile_boxes():
    wl = W.vardiff2d(side=48, tile=16, overlap=6)
    wl["refresh"] = 2
    tol, steps = 1e-6, 5
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    ref = lem_run(X, wl["u0"], wins, steps, "phi", wl["dt"], True, 2, trunc_tol=tol, shape=wl["shape"])
    ctx = L.Lem.from_workload(wl)
    ctx.set_truncation(tol)
    u = torch.tensor(wl["u0"], device="cuda")
    ctx.step(u, steps)
    ctx.sync()
    assert rel_l2(u.cpu().numpy(), ref) <= 1e-12
    # the boxes now in use come from the last rebuild (at step 4, from the state after 4 steps)
    u4 = lem_run(X, wl["u0"], wins, 4, "phi", wl["dt"], True, 2, trunc_tol=tol, shape=wl["shape"])
    J = jacobian(X, u4, wl["dt"], True)
    _check_extents(ctx, wl, tol, lambda ws, t: local_propagators(J, ws, "phi", tiles=[t])[t])
    ctx.close()


def test_zero_tolerance_equals_the_dense_path():
    wl = W.advdiff2d(side=64, tile=16, overlap=8, nu=1.0, a=(1.0, 0.5), dt=1.0, ell=4.0)
    dense = L.Lem.from_workload(wl)
    band = L.Lem.from_workload(wl)
    band.set_truncation(0.0)
    a = torch.tensor(wl["u0"], device="cuda")
    b = torch.tensor(wl["u0"], device="cuda")
    dense.step(a, 10)
    band.step(b, 10)
    torch.cuda.synchronize()
    assert rel_l2(b.cpu().numpy(), a.cpu().numpy()) <= 1e-13
    ext, nv = band.band(0)
    # phi_1 of this local operator is positive everywhere, so the box spans the whole
    # 32 x 32 window from every owner (offsets 8..23 from either edge)
    assert ext == (23, 23, 23, 23) and nv == 32 * 32
    band.set_truncation(-1.0)  # off again: the path lem_create chose
    assert L.APPLY_PATHS[band.info()["apply_path"]] == L.APPLY_PATHS[dense.info()["apply_path"]]
    dense.close()
    band.close()


def test_truncation_refusals():
    wl = W.schrodinger1d()
    ctx = L.Lem.from_workload(wl)
    with pytest.raises(L.LemError) as e:
        ctx.set_truncation(1e-8)
    assert e.value.status == L.LEM_EINVAL
    ctx.close()
    wl = W.heat1d(n=256, tile=32, overlap=8, mu=2.0)
    ctx = L.Lem.from_workload(wl)
    with pytest.raises(L.LemError):
        ctx.band(0)  # no truncation set
    ctx.set_truncation(1e-8)
    with pytest.raises(L.LemError) as e:
        ctx.band(0)  # not built
    assert e.value.status == L.LEM_ENOTREADY
    ctx.build()
    u = torch.tensor(wl["u0"], device="cuda")
    with pytest.raises(L.LemError) as e:
        ctx.step_noalloc(u, 1)
    assert e.value.status == L.LEM_EINVAL
    ctx.close()
