"""Serving layer (lem_server_*): continuous batching of independent requests.

Each request's result must not depend on what else runs: every request, on every tier, is
bit-identical in a mix and alone (one lem_step call of all its steps). The FP64 tier runs the
same kernels on the same inputs. The split tier advances in chunks of a few steps, two of the
requests on one shared context, but each request keeps its float-float state resident and
carries the residual scale from chunk to chunk, so the chunk boundaries change nothing. The
FP64 tier also matches the oracle. The budget queues requests instead of failing them; a
request that can never fit, a host-injected allocation failure and an expired bounded wait
each report their status."""
import os
import time

import numpy as np
import pytest

from oracle import assemble_operator, decompose, lem_run, rel_l2
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


def _requests():
    out = []
    h = W.heat1d(n=1024)
    out.append((h, 1e-10, 9))
    out.append((W.heat1d(n=4096, tile=64, overlap=16, seed=5), 1e-6, 12))  # 1D at 1e-6: no tensor path, FP64
    out.append((W.advdiff2d(side=512, ell=8.0, seed=6), 1e-6, 7))          # split path
    out.append((W.advdiff2d(side=160, ell=8.0, seed=7), 1e-6, 5))          # split path, ragged blocks
    out.append((W.advdiff2d(side=256, tile=16, overlap=4, ell=8.0, seed=8), 1e-10, 6))  # FP64 tier
    out.append((W.advdiff2d(side=512, ell=8.0, seed=9), 1e-6, 3))          # shares the 512^2 context
    return out


def _alone(wl, tol, steps):
    """The same request advanced alone, with the server's precision rule."""
    ctx = L.Lem.from_workload(wl, prec="split" if tol >= 1e-6 else "fp64")
    path = L.APPLY_PATHS[ctx.info()["apply_path"]]
    h = wl["u0"].copy()
    ctx.step_host(h, steps)
    ctx.close()
    return h, path


def test_results_identical_alone_and_in_the_mix():
    reqs = _requests()
    srv = L.Server()
    states = [wl["u0"].copy() for wl, _, _ in reqs]
    tickets = [srv.submit(wl["shape"], wl["bc"], wl["coef"], wl["dt"], wl["tile"], wl["overlap"], st, n, tol)
               for (wl, tol, n), st in zip(reqs, states)]
    for t in tickets:
        srv.wait(t, 120.0)
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["ctx_hits"] >= 1  # the two 512^2 requests share propagators
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    paths = set()
    for (wl, tol, n), st in zip(reqs, states):
        alone, path = _alone(wl, tol, n)
        paths.add(path)
        assert np.array_equal(st, alone), (wl["name"], path)
    assert "tc_split" in paths and "fp64_gemm" in paths
    # FP64 tier against the oracle
    wl, tol, n = reqs[0]
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    ref = lem_run(X, wl["u0"], decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"]), n)
    assert rel_l2(states[0], ref) <= 1e-12


def test_budget_queues_instead_of_failing():
    # different dt -> different propagators; the budget holds about one context at a time
    srv = L.Server(budget_bytes=int(80e6))  # one context (~54 MB incl. build scratch) at a time
    states, tickets = [], []
    for k in range(4):
        wl = W.advdiff2d(side=256, tile=16, overlap=4, ell=8.0, dt=1.0 + 0.5 * k, seed=20 + k)
        st = wl["u0"].copy()
        states.append((wl, st))
        tickets.append(srv.submit(wl["shape"], wl["bc"], wl["coef"], wl["dt"], wl["tile"], wl["overlap"], st, 3,
                                  1e-10))
    for t in tickets:
        srv.wait(t, 120.0)
    s = srv.stats()
    srv.close()
    assert s["completed"] == 4 and s["failed"] == 0 and s["ctx_misses"] == 4
    for wl, st in states:
        assert np.array_equal(st, _alone(wl, 1e-10, 3)[0])


def test_request_larger_than_budget_is_rejected():
    srv = L.Server(budget_bytes=1 << 20)
    wl = W.advdiff2d(side=256, tile=16, overlap=4, ell=8.0)
    st = wl["u0"].copy()
    t = srv.submit(wl["shape"], wl["bc"], wl["coef"], wl["dt"], wl["tile"], wl["overlap"], st, 2, 1e-10)
    with pytest.raises(L.LemError) as e:
        srv.wait(t, 30.0)
    assert e.value.status == L.LEM_ENOMEM
    assert np.array_equal(st, wl["u0"])  # untouched
    srv.close()


def test_bounded_wait_times_out_then_completes():
    srv = L.Server()
    wl = W.advdiff2d(side=1024, ell=8.0)
    st = wl["u0"].copy()
    t = srv.submit(wl["shape"], wl["bc"], wl["coef"], wl["dt"], wl["tile"], wl["overlap"], st, 40, 1e-10)
    with pytest.raises(L.LemError) as e:
        srv.wait(t, 1e-4)
    assert e.value.status == L.LEM_ETIMEOUT
    srv.wait(t, 300.0)
    assert srv.poll(t)
    srv.close()


def test_injected_allocation_failure_reports_enomem():
    srv = L.Server()
    wl = W.heat1d(n=512, tile=64, overlap=8)
    st = wl["u0"].copy()
    os.environ["LEM_FAULT"] = "alloc"
    try:
        t = srv.submit(wl["shape"], wl["bc"], wl["coef"], wl["dt"], wl["tile"], wl["overlap"], st, 2, 1e-10)
        deadline = time.time() + 30
        while srv.status(t) == L.LEM_OK and not srv.poll(t) and time.time() < deadline:
            time.sleep(0.01)
    finally:
        del os.environ["LEM_FAULT"]
    assert srv.status(t) == L.LEM_ENOMEM
    srv.close()


def test_propagator_shared_across_mesh_sizes():
    """Periodic problems with the same stencil, dt, tile and overlap have the same local
    operator whatever the mesh size: a new context takes the cached propagator instead of
    building it, and its result is exactly the one of a context that built its own."""
    srv = L.Server()
    a = W.advdiff2d(side=256, ell=8.0, seed=11)
    b = W.advdiff2d(side=384, ell=8.0, seed=12)
    sa, sb = a["u0"].copy(), b["u0"].copy()
    ta = srv.submit(a["shape"], a["bc"], a["coef"], a["dt"], a["tile"], a["overlap"], sa, 3, 1e-10)
    srv.wait(ta, 120.0)
    tb = srv.submit(b["shape"], b["bc"], b["coef"], b["dt"], b["tile"], b["overlap"], sb, 4, 1e-10)
    srv.wait(tb, 120.0)
    st = srv.stats()
    srv.close()
    assert st["ctx_adopted"] == 1 and st["ctx_misses"] == 2
    assert np.array_equal(sb, _alone(b, 1e-10, 4)[0])
