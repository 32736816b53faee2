"""Anisotropic tiles and windows (tile and overlap chosen per axis; Sec. 1, Sec. 4.3: a
column-wise decomposition for a high vertical Courant number) on every apply path, against
the FP64 oracle: the FP64 GEMM and GEMV paths within 1e-12, the tensor-core split tiers within
the 1e-6 bar."""
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


_REF = {}


def _run(wl, prec, steps):
    key = (wl["name"], wl["tile"], wl["overlap"], steps)
    if key not in _REF:
        X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
        wins = decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
        _REF[key] = lem_run(X, wl["u0"], wins, steps, "phi", wl["dt"], wl.get("reaction", False),
                            wl.get("refresh", 0))
    ref = _REF[key]
    ctx = L.Lem.from_workload(wl, prec=prec)
    u = torch.tensor(wl["u0"], dtype=torch.float64, device="cuda")
    ctx.step(u, steps)
    ctx.sync()
    path = L.APPLY_PATHS[ctx.info()["apply_path"]]
    ctx.close()
    return rel_l2(u.cpu().numpy(), ref), path


def test_tall_windows_fp64():
    wl = W.advdiff2d(side=64, tile=(16, 16), overlap=(12, 4), a=(0.125, 1.5))
    err, path = _run(wl, "fp64", 10)
    assert path == "fp64_gemm" and err <= 1e-12


def test_column_strips_whole_axis_fp64():
    """Whole columns: windows wrap the periodic vertical axis (no vertical overlap)."""
    wl = W.advdiff2d(side=64, tile=(64, 8), overlap=(0, 4), a=(0.125, 1.5))
    err, path = _run(wl, "fp64", 10)
    assert err <= 1e-12


def test_ragged_rectangular_dirichlet_variable_fp64_gemv():
    """Rectangular tiles that do not divide the mesh, clipped at Dirichlet walls, per-tile
    propagators (variable coefficients): the batched GEMV."""
    wl = W.vardiff2d(side=60, tile=12, overlap=5)
    wl["tile"], wl["overlap"] = (12, 20), (5, 3)
    err, path = _run(wl, "fp64", 4)
    assert path == "fp64_gemv" and err <= 1e-12


@pytest.mark.parametrize("prec", ["split", "split_fast"])
def test_tall_windows_tensor_split(prec):
    """Tiles 32 x 16 with overlap 16 x 8: windows 64 x 32, a K of 64 window rows of 32."""
    wl = W.advdiff2d(side=256, tile=(32, 16), overlap=(16, 8), a=(0.25, 1.5))
    err, path = _run(wl, prec, 20)
    print(f"{prec}: tall windows 64 x 32 on 256^2, 20 steps: rel_l2 {err:.2e}")
    assert path == "tc_split" and err <= 1e-6
