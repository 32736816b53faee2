"""Failure detection without a GPU fault, and checkpointing of propagators.

* A tensor-core kernel whose mbarrier wait runs out (LEM_FAULT=timeout: one CTA arms a stage
  whose bytes never come) gives up after its bounded wait, the host reads LEM_ETIMEOUT, and the
  CUDA context stays usable for other contexts.
* A refused admission (LEM_FAULT=admit, host side) fails the request with its status.
* Propagators exported with lem_get_propagator and loaded into a fresh context with
  lem_set_propagators reproduce the original steps bit for bit (the checkpoint story: the state
  is the caller's buffer, the propagators round-trip through host memory)."""
import numpy as np
import pytest

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


def test_bounded_device_wait_reports_timeout_and_context_survives(monkeypatch):
    wl = W.advdiff2d(side=256, ell=8.0, seed=21)
    monkeypatch.setenv("LEM_FAULT", "timeout")
    bad = L.Lem.from_workload(wl, prec="split")
    monkeypatch.delenv("LEM_FAULT")
    assert bad.info()["split_path"] == 1
    u = torch.tensor(wl["u0"], device="cuda")
    bad.step(u, 1)
    with pytest.raises(L.LemError) as e:
        bad.sync()
    assert e.value.status == L.LEM_ETIMEOUT
    bad.sync()  # the error was reported once and cleared; the stream is healthy
    bad.close()
    # the device and other contexts are unaffected
    good = L.Lem.from_workload(wl, prec="split")
    ref = L.Lem.from_workload(wl, prec="split")
    a = torch.tensor(wl["u0"], device="cuda")
    b = torch.tensor(wl["u0"], device="cuda")
    good.step(a, 3)
    ref.step(b, 3)
    good.sync()
    ref.sync()
    assert torch.equal(a, b) and torch.isfinite(a).all()


def test_refused_admission_fails_the_request(monkeypatch):
    wl = W.advdiff2d(side=128, ell=8.0, seed=22)
    srv = L.Server()
    monkeypatch.setenv("LEM_FAULT", "admit")
    st = wl["u0"].copy()
    t = srv.submit(wl["shape"], wl["bc"], wl["coef"], wl["dt"], wl["tile"], wl["overlap"], st, 2, 1e-10)
    with pytest.raises(L.LemError) as e:
        srv.wait(t, 60.0)
    assert e.value.status == L.LEM_ENOMEM
    monkeypatch.delenv("LEM_FAULT")
    t2 = srv.submit(wl["shape"], wl["bc"], wl["coef"], wl["dt"], wl["tile"], wl["overlap"], st, 2, 1e-10)
    srv.wait(t2, 120.0)
    assert srv.stats()["failed"] == 1
    srv.close()


@pytest.mark.parametrize("wl_name,prec", [("heat1d", "fp64"), ("advdiff2d", "split"), ("vardiff2d", "fp64")])
def test_propagators_round_trip_through_host(wl_name, prec):
    wl = {"heat1d": W.heat1d(n=512, tile=32, overlap=8),
          "advdiff2d": W.advdiff2d(side=256, ell=8.0, seed=23),
          "vardiff2d": W.vardiff2d(side=64, tile=16, overlap=4)}[wl_name]
    wl["reaction"] = False
    src = L.Lem.from_workload(wl, prec=prec)
    src.build()
    inf = src.info()
    P = np.stack([src.propagator(c) for c in range(inf["nclasses"])])
    sq = [src.squarings(c) for c in range(inf["nclasses"])]
    dst = L.Lem.from_workload(wl, prec=prec)
    dst.set_propagators(P, sq)
    assert dst.info()["built"] == 1 and dst.squarings(0) == sq[0]
    a = torch.tensor(wl["u0"], device="cuda")
    b = torch.tensor(wl["u0"], device="cuda")
    src.step(a, 4)
    dst.step(b, 4)
    src.sync()
    dst.sync()
    assert torch.equal(a, b)
