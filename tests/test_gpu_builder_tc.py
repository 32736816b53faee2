"""Propagators built with the tensor-core products (split-precision tiers) against the FP64
oracle's Pade-13 phi_1 / exp (Sec. 3 step 2, Sec. 4) and against the FP64 GPU build.

The split tiers build every matrix product of the Pade evaluation and of the squarings as an
exact sum of FP16 slice products (7 slices of 7 bits per operand, row / column power-of-two
scales, exact FP32 integer partial sums over K chunks of 128, float-float accumulation). One
product then carries an error below about n 2^-48 max|A_i,:| max|B_:,j| per entry; the
propagator stays within TOL_TC of max|P| after up to a dozen products and the squarings.
The bar: 1e-11 of max|P| elementwise, far below what the FP16-piece apply can resolve."""
import os

import numpy as np
import pytest

from oracle import assemble_operator, decompose, jacobian, local_propagators
from paper_1505_02248_gb300 import lem as L
from paper_1505_02248_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_TC = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_02248_gb300 import build as B
    B.build()
    L.load()


def _classes(ctx, nwin, limit):
    seen = {}
    for t in range(nwin):
        c = ctx.tile_class(t)
        if c not in seen:
            seen[c] = t
        if len(seen) >= limit:
            break
    return seen


def _compare(wl, prec, mode="phi", limit=6):
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    wins = decompose(wl["shape"], wl["bc"], wl["tile"], wl["overlap"])
    Xj = jacobian(X, wl["u0"], wl["dt"], True) if wl.get("reaction") else X
    tc = L.Lem.from_workload(wl, prec=prec, mode=mode)
    f64 = L.Lem.from_workload(wl, prec="fp64", mode=mode)
    u = torch.tensor(wl["u0"], dtype=torch.float64, device="cuda")
    tc.build(u)
    f64.build(u)
    worst_oracle = worst_f64 = 0.0
    sq = []
    for c, t in _classes(tc, len(wins), limit).items():
        P_ref = local_propagators(Xj, wins, mode, tiles=[t])[t]
        ni, nl = P_ref.shape
        P = tc.propagator(c)
        Pf = f64.propagator(f64.tile_class(t))
        scale = np.abs(P_ref).max()
        worst_oracle = max(worst_oracle, np.abs(P[:ni, :nl] - P_ref).max() / scale)
        worst_f64 = max(worst_f64, np.abs(P - Pf).max() / scale)
        assert not P[:ni, nl:].any() and not P[ni:, :].any()  # zero padding stays zero
        assert tc.squarings(c) == f64.squarings(f64.tile_class(t))
        sq.append(tc.squarings(c))
    tc.close()
    f64.close()
    return worst_oracle, worst_f64, sq


@pytest.mark.parametrize("mode", ["phi", "exp"])
def test_heat1d_tc_build(mode):
    wl = W.heat1d(n=256, tile=64, overlap=16)
    eo, ef, _ = _compare(wl, "split", mode)
    print(f"heat1d {mode}: vs oracle {eo:.2e}, vs fp64 build {ef:.2e}")
    assert eo <= TOL_TC and ef <= TOL_TC


@pytest.mark.parametrize("mode", ["phi", "exp"])
def test_advdiff2d_shared_window_tc_build(mode):
    """48 x 48 windows (n = 2304: 18 exact K chunks per product)."""
    wl = W.advdiff2d(side=256)
    eo, ef, _ = _compare(wl, "split", mode, limit=1)
    print(f"advdiff2d {mode}: vs oracle {eo:.2e}, vs fp64 build {ef:.2e}")
    assert eo <= TOL_TC and ef <= TOL_TC


def test_per_tile_reaction_tc_build_uneven_squarings():
    """Per-tile propagators (variable k, u - u^3 Jacobian), windows clipped at the walls (a
    zero-padded frame), and squaring counts that differ between classes of one batch: the
    squarings then run on a prefix of the classes sorted by count."""
    wl = W.vardiff2d(side=96, tile=16, overlap=6)
    wl["coef"] = {k: v * np.where(np.arange(96 * 96).reshape(96, 96) % 96 < 48, 1.0, 6.0)
                  for k, v in wl["coef"].items()}
    eo, ef, sq = _compare(wl, "split_fast", limit=40)
    print(f"vardiff per tile: vs oracle {eo:.2e}, vs fp64 build {ef:.2e}, squarings {sorted(set(sq))}")
    assert len(set(sq)) > 1
    assert eo <= TOL_TC and ef <= TOL_TC


def test_fp64_products_switch_reproduces_fp64_build(monkeypatch):
    """LEM_BUILD_PRODUCTS=fp64 builds split-tier propagators with the FP64 GEMM: bit for bit
    the FP64 tier's propagators."""
    monkeypatch.setenv("LEM_BUILD_PRODUCTS", "fp64")
    wl = W.advdiff2d(side=128)
    a = L.Lem.from_workload(wl, prec="split")
    b = L.Lem.from_workload(wl, prec="fp64")
    a.build()
    b.build()
    assert np.array_equal(a.propagator(0), b.propagator(0))
    a.close()
    b.close()
