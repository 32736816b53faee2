"""The allocation-free FP64 step (lem_step_fp64_noalloc) against the ordinary step.

lem_step_fp64_noalloc serves callers that must not allocate device memory while stepping
(runtimes that own all device memory through their own pool, loops that cannot take
cudaMalloc's synchronisation); its scratch is a static device array. Here it must give the
same state as lem_step within the FP64 tolerance of the other parity tests, on two calls in a
row (the second call reuses the array the first one left behind), on both apply paths it
takes (one gathered GEMM per propagator class, and the batched GEMV for problems with a
propagator per tile), and must refuse problems larger than its scratch. This file is
collected last so that a stop-at-first-failure run has already run every other test."""
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


def _case(case):
    if case == "heat1d":  # 16 tiles in 3 classes: lem_create picks the batched GEMV
        return W.heat1d(), "fp64_gemv"
    if case == "advdiff2d_128":  # 64 tiles, one shared propagator: the gathered GEMM
        return W.advdiff2d(side=128, tile=16, overlap=4, ell=8.0), "fp64_gemm"
    wl = W.vardiff2d(side=96, tile=16, overlap=6)  # a propagator per tile: the batched GEMV
    if case == "vardiff2d_96_linear":
        wl["reaction"] = False
    return wl, "fp64_gemv"


@pytest.mark.parametrize("case", ["heat1d", "advdiff2d_128", "vardiff2d_96_reaction", "vardiff2d_96_linear"])
def test_noalloc_matches_lem_step_on_two_calls(case):
    wl, path = _case(case)
    ref_ctx = L.Lem.from_workload(wl)
    na_ctx = L.Lem.from_workload(wl)
    u_ref = torch.tensor(wl["u0"], device="cuda")
    u_na = torch.tensor(wl["u0"], device="cuda")
    na_ctx.build(u_na)  # the reaction's Jacobian is taken at u0, as lem_step's first build does
    assert L.APPLY_PATHS[na_ctx.info()["apply_path"]] == path
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
