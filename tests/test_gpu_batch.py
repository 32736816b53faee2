"""GPU checks of the batch layer (lem_batch_*): many independent problems of uneven size
advanced by one CUDA graph launch. The local problems of the method are independent
(Sec. 3), so a batch must give each problem exactly what its own lem_step calls give, and
that in turn matches the FP64 oracle within the bar of the problem's precision."""
import numpy as np
import pytest

from oracle import assemble_operator, decompose, lem_run, rel_l2
from paper_1505_02248_gb300 import lem as L
from paper_1505_02248_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_SPLIT = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_02248_gb300 import build as B
    B.build()
    L.load()


def _problems():
    probs = W.batch_problems(n=20, seed=5, side_max=128)
    for p in probs:
        p["prec"] = "split"
    # a 1D Dirichlet problem on the FP64 path and a 2D one on the FP64 GEMV path ride along
    h1 = W.heat1d(n=256, tile=32, overlap=8)
    h1["prec"] = "fp64"
    v2 = W.vardiff2d(side=64, tile=16, overlap=4)
    v2["reaction"] = False
    v2["prec"] = "fp64"
    return probs + [h1, v2]


def _ctx(p):
    return L.Lem.from_workload(p, prec=p["prec"])


@pytest.mark.parametrize("steps_per_launch,launches,lanes", [(2, 3, 4), (1, 2, 1), (4, 1, 16)])
def test_batch_equals_per_problem_steps(steps_per_launch, launches, lanes):
    probs = _problems()
    # per-problem reference through lem_step with the same call boundaries
    ref = []
    for p in probs:
        c = _ctx(p)
        u = torch.tensor(p["u0"], device="cuda")
        for _ in range(launches):
            c.step(u, steps_per_launch)
        c.sync()
        ref.append(u.cpu().numpy())
        c.close()
    ctxs = [_ctx(p) for p in probs]
    states = [torch.tensor(p["u0"], device="cuda") for p in probs]
    b = L.Batch(ctxs, states, steps_per_launch=steps_per_launch, lanes=lanes)
    torch.cuda.synchronize()
    # creation warms up on copies: the states are untouched
    for p, s in zip(probs, states):
        assert np.array_equal(s.cpu().numpy(), p["u0"])
    b.run(launches)
    torch.cuda.synchronize()
    for i, (s, r) in enumerate(zip(states, ref)):
        assert np.array_equal(s.cpu().numpy(), r), probs[i]["name"]
    est, lane = b.schedule()
    cands = b.candidates()
    chosen = [c for c in cands if c["chosen"]]
    assert len(chosen) == 1 and all(c["ms"] > 0 for c in cands)
    # the autotuner tried lanes/2, lanes and 2 lanes (within 1..n)
    want = sorted({max(1, min(k, len(probs))) for k in (lanes // 2, lanes, 2 * lanes)})
    assert sorted(c["lanes"] for c in cands if not c["fused"]) == want
    if not chosen[0]["fused"]:
        nl = chosen[0]["lanes"]
        assert np.all(est > 0) and lane.min() >= 0 and lane.max() < nl
        # longest-processing-time bound on the busiest lane
        loads = np.bincount(lane, weights=est, minlength=nl)
        assert loads.max() <= est.sum() / nl + est.max() + 1e-9
    b.close()


def test_batch_vs_oracle():
    probs = [p for p in _problems()[:20] if p["shape"][0] <= 96][:4]
    ctxs = [_ctx(p) for p in probs]
    states = [torch.tensor(p["u0"], device="cuda") for p in probs]
    b = L.Batch(ctxs, states, steps_per_launch=4, lanes=4)
    b.run(2)
    torch.cuda.synchronize()
    for p, s in zip(probs, states):
        X = assemble_operator(p["shape"], p["bc"], p["coef"], p["dt"])
        wins = decompose(p["shape"], p["bc"], p["tile"], p["overlap"])
        ref = lem_run(X, p["u0"], wins, 8)
        err = rel_l2(s.cpu().numpy(), ref)
        print(f"{p['name']}: rel_l2 {err:.3e}")
        assert err <= TOL_SPLIT, p["name"]


def test_batch_rejects_bad_arguments():
    p = _problems()[0]
    c = _ctx(p)
    s = torch.tensor(p["u0"], device="cuda")
    with pytest.raises(L.LemError):
        L.Batch([c], [s], steps_per_launch=0)
    with pytest.raises(L.LemError):
        L.Batch([c], [s], lanes=0)
    v = W.vardiff2d(side=64, tile=16, overlap=4)
    v["refresh"] = 2
    cr = L.Lem.from_workload(v)
    sr = torch.tensor(v["u0"], device="cuda")
    with pytest.raises(L.LemError):
        L.Batch([cr], [sr])


@pytest.mark.parametrize("schedule", ["fused:0", "fused:128", "fused:64", "fused:32", "lanes"])
def test_split_batch_schedules_equal_per_problem_steps(schedule, monkeypatch):
    """All-split batches can run fused (one residual and one persistent GEMM launch per step
    for every problem; every window-block width cap the autotuner tries) or on lanes; each
    gives each problem exactly its own lem_step result."""
    monkeypatch.setenv("LEM_BATCH_SCHEDULE", schedule)
    probs = W.batch_problems(n=24, seed=7, side_max=160)
    ref = []
    for p in probs:
        c = L.Lem.from_workload(p, prec="split")
        u = torch.tensor(p["u0"], device="cuda")
        for _ in range(2):
            c.step(u, 3)
        c.sync()
        ref.append(u.cpu().numpy())
        c.close()
    ctxs = [L.Lem.from_workload(p, prec="split") for p in probs]
    states = [torch.tensor(p["u0"], device="cuda") for p in probs]
    b = L.Batch(ctxs, states, steps_per_launch=3, lanes=4)
    info = b.info()
    assert info["fused_ms"] > 0 and info["lanes_ms"] > 0
    assert info["fused"] == schedule.startswith("fused")
    chosen = [c for c in b.candidates() if c["chosen"]][0]
    if info["fused"]:
        assert chosen["n_cap"] == int(schedule.split(":")[1])
        alg, exe = b.gemm_work()
        assert exe >= alg > 0
    b.run(2)
    b.sync()
    for i, (s, r) in enumerate(zip(states, ref)):
        assert np.array_equal(s.cpu().numpy(), r), probs[i]["name"]
    print(f"{schedule}: lanes {info['lanes_ms']:.3f} ms, fused {info['fused_ms']:.3f} ms per launch")
    b.close()
