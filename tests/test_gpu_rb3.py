"""The third-order exponential Rosenbrock scheme (exprb32; Sec. 4.2 runs its nonlinear tests
with a third-order exponential Rosenbrock method) on the GPU against the oracle: the phi_1 and
phi_3 propagators built together (FP64 products, and tensor-core slice products for the split
tiers), and the two-stage LEM step on the batched GEMV (FP64, and FP32 propagators).

Bars: propagators within 1e-11 of max|P| (the GPU evaluates Pade-13 on the augmented matrix with
unit identity blocks and undoes the scaling with phi doubling steps, the oracle squares the scaled
augmented matrix: both to about unit roundoff); FP64 steps within 1e-12 relative L2; the FP32
tier within 1e-6."""
import numpy as np
import pytest

from oracle import assemble_operator, decompose, jacobian, lem_run_rb3, local_propagators, rel_l2
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


def _case(side=40, tile=8, H=3, refresh=2):
    wl = W.vardiff2d(side=side, tile=tile, overlap=H)
    wl["refresh"] = refresh
    return wl


@pytest.mark.parametrize("prec", ["fp64", "split_fast"])
def test_phi1_phi3_propagators(prec):
    wl = _case()
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    J = jacobian(X, wl["u0"], wl["dt"], True)
    ctx = L.Lem.from_workload(wl, prec=prec, scheme="rb3")
    u = torch.tensor(wl["u0"], dtype=torch.float64, device="cuda")
    ctx.build(u)
    worst, sq, seen = 0.0, set(), set()
    for t in range(len(wins)):
        c = ctx.tile_class(t)
        if c in seen:
            continue
        seen.add(c)
        sq.add(ctx.squarings(c))
        for get, mode in ((ctx.propagator, "phi"), (ctx.propagator_phi3, "phi3")):
            ref = local_propagators(J, wins, mode, tiles=[t])[t]
            got = get(c)
            ni, nl = ref.shape
            worst = max(worst, np.abs(got[:ni, :nl] - ref).max() / np.abs(ref).max())
            assert not got[:ni, nl:].any() and not got[ni:, :].any()
    ctx.close()
    print(f"{prec}: phi_1/phi_3 vs oracle {worst:.2e} over {len(seen)} classes, squarings {sorted(sq)}")
    assert len(sq) > 1 and worst <= 1e-11


@pytest.mark.parametrize("prec,bar", [("fp64", 1e-12), ("split_fast", 1e-6)])
def test_rb3_steps_vs_oracle(prec, bar):
    wl = _case()
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    steps = 6
    ref = lem_run_rb3(X, wl["u0"], wins, steps, wl["dt"], refresh=wl["refresh"])
    ctx = L.Lem.from_workload(wl, prec=prec, scheme="rb3")
    u = torch.tensor(wl["u0"], dtype=torch.float64, device="cuda")
    ctx.step(u, steps)
    ctx.sync()
    path = L.APPLY_PATHS[ctx.info()["apply_path"]]
    ctx.close()
    err = rel_l2(u.cpu().numpy(), ref)
    print(f"{prec} ({path}): rb3 {steps} steps rel_l2 {err:.2e}")
    assert path in ("fp64_gemv", "f32_gemv") and err <= bar


def test_rb3_differs_from_euler_and_needs_phi_mode():
    """The second stage is not a no-op on a nonlinear problem, and the scheme is PHI only."""
    wl = _case()
    a = L.Lem.from_workload(wl, scheme="rb3")
    b = L.Lem.from_workload(wl)
    ua = torch.tensor(wl["u0"], dtype=torch.float64, device="cuda")
    ub = ua.clone()
    a.step(ua, 3)
    b.step(ub, 3)
    a.sync()
    b.sync()
    assert rel_l2(ua.cpu().numpy(), ub.cpu().numpy()) > 1e-6
    a.close()
    b.close()
    wl2 = W.advdiff2d(side=64)
    with pytest.raises(L.LemError):
        L.Lem.from_workload(wl2, mode="exp", scheme="rb3")
