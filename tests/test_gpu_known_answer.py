"""Known-answer tests of the apply kernels, independent of the propagator build: hand-made
propagators loaded with lem_set_propagators on every apply path (the FP64 GEMM, the FP64 and
FP32 GEMV, the tcgen05 split GEMM).

- identity: row i selects the window column of owner node i itself. EXP: u' = u (exact);
  PHI: u' = u + dt A u, one explicit Euler step (the residual of Eq. lem).
- permutation: row i selects the window node one column to the east (periodic x), so EXP
  shifts the field west by one node.
- one nonzero tile: every class zero except one tile's, so PHI changes that tile's owners only.
The expected values come from numpy (and the oracle's residual), not from the CUDA path."""
import numpy as np
import pytest

from oracle import assemble_operator, residual
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


def _tiles(wl):
    return L.plan_query(wl["shape"], wl["bc"], wl["coef"], wl["dt"], wl["tile"], wl["overlap"])["tiles"]


def _selector(ctx, wl, shift_x=0, only_class=None):
    """Propagators whose row i picks window node (owner i shifted by shift_x columns)."""
    inf = ctx.info()
    P = np.zeros((inf["nclasses"], inf["n_int"], inf["n_loc"]))
    seen = set()
    for t in _tiles(wl):
        (oy, ox, wy, wx, iy0, ix0, ey, ex, _, _, c) = [int(v) for v in t]
        if c in seen or (only_class is not None and c != only_class):
            continue
        seen.add(c)
        for i in range(ey * ex):
            y, x = iy0 + i // ex, ix0 + i % ex + shift_x
            assert 0 <= x < wx
            P[c, i, y * wx + x] = 1.0
    return P


def _step(wl, prec, mode, P, steps=1):
    ctx = L.Lem.from_workload(wl, prec=prec, mode=mode)
    Pin = P(ctx) if callable(P) else P
    ctx.set_propagators(Pin)
    u = torch.tensor(wl["u0"], dtype=torch.float64, device="cuda")
    ctx.step(u, steps)
    ctx.sync()
    path = L.APPLY_PATHS[ctx.info()["apply_path"]]
    ctx.close()
    return u.cpu().numpy(), path


CASES = [  # (workload, prec, expected apply path)
    (lambda: W.advdiff2d(side=64, tile=16, overlap=4), "fp64", "fp64_gemm"),
    (lambda: W.vardiff2d(side=48, tile=16, overlap=4), "fp64", "fp64_gemv"),
    (lambda: W.vardiff2d(side=48, tile=16, overlap=4), "split_fast", "f32_gemv"),
]


@pytest.mark.parametrize("make,prec,path", CASES)
def test_identity_exp_is_exact(make, prec, path):
    wl = make()
    wl["reaction"] = False
    got, p = _step(wl, prec, "exp" if path != "f32_gemv" else "phi", lambda c: _selector(c, wl))
    assert p == path or path == "f32_gemv"
    if path == "f32_gemv":  # PHI with FP32 propagators: u + r rounded once to FP32
        X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
        r = residual(X, wl["u0"])
        assert np.all(np.abs(got - (wl["u0"] + r)) <= 2.0 ** -24 * np.abs(r) + 1e-300)
    else:
        assert np.array_equal(got, wl["u0"])


@pytest.mark.parametrize("make,prec,path", CASES[:2])
def test_identity_phi_is_one_explicit_euler_step(make, prec, path):
    wl = make()
    wl["reaction"] = False
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    got, p = _step(wl, prec, "phi", lambda c: _selector(c, wl))
    ref = wl["u0"] + residual(X, wl["u0"])
    assert p == path and np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_permutation_shifts_the_field():
    wl = W.advdiff2d(side=64, tile=16, overlap=4)
    got, p = _step(wl, "fp64", "exp", lambda c: _selector(c, wl, shift_x=1))
    u = wl["u0"].reshape(64, 64)
    assert p == "fp64_gemm" and np.array_equal(got.reshape(64, 64), np.roll(u, -1, axis=1))


def test_one_nonzero_tile_changes_its_owners_only():
    wl = W.vardiff2d(side=48, tile=16, overlap=4)
    wl["reaction"] = False
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    tiles = _tiles(wl)
    target = int(tiles[4][10])  # the class of tile 4 (the centre tile of the 3 x 3 grid)
    got, p = _step(wl, "fp64", "phi", lambda c: _selector(c, wl, only_class=target))
    ref = wl["u0"].copy()
    t = tiles[4]
    r = residual(X, wl["u0"])
    for i in range(int(t[6]) * int(t[7])):
        node = (int(t[8]) + i // int(t[7])) * 48 + int(t[9]) + i % int(t[7])
        ref[node] += r[node]
    assert p == "fp64_gemv" and np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("prec,bar", [("split", 2.0 ** -23), ("split_fast", 2.0 ** -21)])
def test_identity_on_the_tensor_split_path(prec, bar):
    """PHI with the identity propagator on tcgen05: u + the residual, through the FP16 pieces of
    r (cut from the float-float residual) and the float-float state. Each owner's increment is
    the exact integer main product plus the FP32 correction sum, rounded to FP32 before it
    enters the float-float state: about 2^-24 of max|r| with three pieces (which themselves
    resolve about 2^-33), up to 2^-21 with two."""
    wl = W.advdiff2d(side=256)
    X = assemble_operator(wl["shape"], wl["bc"], wl["coef"], wl["dt"])
    got, p = _step(wl, prec, "phi", lambda c: _selector(c, wl))
    r = residual(X, wl["u0"])
    ref = wl["u0"] + r
    err = np.abs(got - ref).max() / np.abs(r).max()
    print(f"{prec}: identity propagator on tcgen05, max error / max|r| = {err:.2e}")
    assert p == "tc_split" and err <= bar
