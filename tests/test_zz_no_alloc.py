"""The allocation-free FP64 step (lem_step_fp64_noalloc) against the ordinary step.

lem_step_fp64_noalloc serves callers that must not allocate device memory while stepping
(stream capture, externally owned memory pools, loops that cannot take cudaMalloc's
synchronisation); its scratch is a static device array. Here it must give the same state as
lem_step within the FP64 tolerance of the other parity tests, on two calls in a row (the
second call reuses the array the first one left behind), and must refuse problems larger
than its scratch. This file is collected last so that a stop-at-first-failure run has
already run every other test."""
import numpy as np
import pytest

from paper_1505_02248_gb300 import lem as L
from paper_1505_02248_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_02248_gb300 import build as B
    B.build()
    L.load()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("case", ["heat1d", "advdiff2d_128"])
def test_noalloc_matches_lem_step_on_two_calls(case):
    wl = W.heat1d() if case == "heat1d" else W.advdiff2d(side=128, tile=16, overlap=4, ell=8.0)
    ref_ctx = L.Lem.from_workload(wl)
    na_ctx = L.Lem.from_workload(wl)
    na_ctx.build()
    u_ref = torch.tensor(wl["u0"], device="cuda")
    u_na = torch.tensor(wl["u0"], device="cuda")
    for _ in range(2):  # two calls in a row share (and reuse) the static scratch
        ref_ctx.step(u_ref, 7)
        na_ctx.step_noalloc(u_na, 7)
        torch.cuda.synchronize()
        assert _rel(u_na.cpu().numpy(), u_ref.cpu().numpy()) <= TOL


def test_noalloc_rejects_oversized_and_unbuilt_problems():
    big = W.advdiff2d(side=1024, tile=32, overlap=8, ell=8.0)  # 8 MiB residual alone
    ctx = L.Lem.from_workload(big)
    ctx.build()
    u = torch.zeros(big["u0"].size, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LemError) as e:
        ctx.step_noalloc(u, 1)
    assert e.value.status == L.LEM_EINVAL and "bytes" in str(e.value)
    small = W.heat1d(n=128, tile=32, overlap=4)
    c2 = L.Lem.from_workload(small)
    v = torch.tensor(small["u0"], device="cuda")
    with pytest.raises(L.LemError) as e2:
        c2.step_noalloc(v, 1)
    assert e2.value.status == L.LEM_ENOTREADY
