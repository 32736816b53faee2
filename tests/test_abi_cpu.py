"""CPU checks of the C-ABI library: it builds, loads, exports every entry point declared in
include/*.h, validates descriptors, and its host planner reproduces the oracle's
decomposition (Sec. 3: owner tiles D_i, windows M_i). No compute call needs a GPU here."""
import glob
import os
import re

import numpy as np
import pytest

from oracle import decompose
from paper_1505_02248_gb300 import build as B
from paper_1505_02248_gb300 import lem as L
from paper_1505_02248_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(lem_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol(lib):
    declared = _declared()
    assert {"lem_create", "lem_step", "lem_build_propagators"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    # the binding wraps every declared entry point
    assert declared <= {s[0] for s in L.SIGNATURES}


def test_status_strings(lib):
    assert lib.lem_status_str(0) == b"LEM_OK"
    assert lib.lem_status_str(7) == b"LEM_ENUMERIC"


@pytest.mark.parametrize("bad", ["ndim", "n", "tile", "overlap", "dt", "mode", "exp_reaction",
                                 "coef", "refresh", "reaction_kind", "porous_m", "porous_m_nan",
                                 "porous_rb3", "porous_exp"])
def test_invalid_descriptors_rejected(lib, bad):
    coef = W.stencil_advdiff_2d(1.0, 1.0, 0.5, 1.0)
    kw = dict(shape=(64, 64), bc=("periodic", "periodic"), coef=coef, dt=1.0, tile=(16, 16),
              overlap=(4, 4))
    d, keep = L.make_desc(**kw)
    if bad == "ndim":
        d.ndim = 3
    elif bad == "n":
        d.n[0] = 0
    elif bad == "tile":
        d.tile[1] = 0
    elif bad == "overlap":
        d.overlap[0] = -1
    elif bad == "dt":
        d.dt = float("nan")
    elif bad == "mode":
        d.mode = 5
    elif bad == "exp_reaction":
        d.mode, d.reaction = 1, 1
    elif bad == "coef":
        d.coef[3] = L.C.POINTER(L.C.c_double)()
    elif bad == "refresh":
        d.refresh = -2
    elif bad == "reaction_kind":
        d.reaction = 3
    elif bad == "porous_m":
        d.reaction, d.porous_m = 2, 1.0
    elif bad == "porous_m_nan":
        d.reaction, d.porous_m = 2, float("nan")
    elif bad == "porous_rb3":
        d.reaction, d.porous_m, d.scheme = 2, 3.0, 1
    elif bad == "porous_exp":
        d.reaction, d.porous_m, d.mode = 2, 3.0, 1
    st = lib.lem_plan_query(L.C.byref(d), None, None, None, None, None)
    assert st == L.LEM_EINVAL
    assert len(lib.lem_last_error()) > 0


@pytest.mark.parametrize("shape,bc,tile,H", [
    ((1024,), ("dirichlet",), (64,), (16,)),
    ((100,), ("periodic",), (32,), (5,)),
    ((70,), ("dirichlet",), (32,), (3,)),
    ((37, 45), ("dirichlet", "periodic"), (16, 16), (4, 6)),
    ((24, 24), ("periodic", "periodic"), (8, 8), (8, 8)),
    ((2048, 2048), ("periodic", "periodic"), (32, 32), (8, 8)),
])
def test_planner_matches_oracle_decomposition(lib, shape, bc, tile, H):
    coef = {k: 1.0 for k in "CWESN"}
    q = L.plan_query(shape, bc, coef, 1.0, tile, H)
    wins = decompose(shape, bc, tile, H)
    assert q["ntiles"] == len(wins)
    nx = shape[-1]
    ny = shape[0] if len(shape) == 2 else 1
    step = max(1, len(wins) // 64)
    for i in range(0, len(wins), step):
        o = q["tiles"][i]
        oy, ox, wy, wx, iy, ix, ey, ex, ty, tx = (int(v) for v in o[:10])
        M = np.array([((oy + a) % ny) * nx + (ox + b) % nx for a in range(wy) for b in range(wx)])
        D = np.array([(ty + a) * nx + tx + b for a in range(ey) for b in range(ex)])
        assert np.array_equal(M, wins[i].M)
        assert np.array_equal(D, wins[i].D)
        dpos = np.array([(iy + a) * wx + ix + b for a in range(ey) for b in range(ex)])
        assert np.array_equal(dpos, wins[i].d_pos)
    assert q["n_loc"] == max(len(w.M) for w in wins)
    assert q["n_int"] == max(len(w.D) for w in wins)


def test_constant_coefficient_classes(lib):
    coef = W.stencil_heat_1d(1.0, 1.0)
    q = L.plan_query((1024,), ("dirichlet",), coef, 1.0, (64,), (16,))
    assert q["nclasses"] == 3  # left wall, interior, right wall
    coef2 = W.stencil_advdiff_2d(5.0, 1.0, 0.5, 1.0)
    q2 = L.plan_query((2048, 2048), ("periodic", "periodic"), coef2, 4.0, (32, 32), (8, 8))
    assert q2["nclasses"] == 1 and q2["n_loc"] == 2304 and q2["n_int"] == 1024
    kfield = np.ones((64, 64))
    q3 = L.plan_query((64, 64), ("dirichlet", "dirichlet"), W.stencil_vardiff_2d(kfield, 1.0),
                      1.0, (16, 16), (6, 6))
    assert q3["nclasses"] == q3["ntiles"] == 16  # variable coefficients: one class per tile


def test_server_create_without_device_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = L.C.c_void_p()
    st = lib.lem_server_create(0, 0, L.C.byref(h))
    assert st in (L.LEM_ECUDA, L.LEM_EINVAL) and not h.value


def test_porous_descriptor_accepted_with_per_tile_classes(lib):
    """The porous-medium problem (reaction 2) validates on the host; its Jacobian depends on
    the state, so every tile gets its own propagator class."""
    wl = W.porous1d(n=400)
    q = L.plan_query(wl["shape"], wl["bc"], wl["coef"], wl["dt"], wl["tile"], wl["overlap"],
                     porous_m=wl["porous_m"])
    assert q["ntiles"] == 10 and q["nclasses"] == 10
    d, keep = L.make_desc(wl["shape"], wl["bc"], wl["coef"], wl["dt"], wl["tile"], wl["overlap"],
                          porous_m=3.0)
    assert d.reaction == 2 and d.porous_m == 3.0


class _FakeCudaTensor:
    """Just the tensor attributes the binding's checks read (no CUDA device here)."""

    def __init__(self, n, itemsize=8, complex_=False, floating=True, contiguous=True, index=0):
        import torch
        self.is_cuda = True
        self._n, self._contig, self._cplx, self._float = n, contiguous, complex_, floating
        self.dtype = type("D", (), {"itemsize": itemsize})()
        self.device = torch.device("cuda", index)

    def is_contiguous(self):
        return self._contig

    def is_complex(self):
        return self._cplx

    def is_floating_point(self):
        return self._float

    def numel(self):
        return self._n


def test_device_state_checks_raise_instead_of_passing_bad_pointers():
    """The binding hands the library a raw device pointer: a host tensor, a wrong type or size,
    or another device must raise (explicit checks, kept under python -O)."""
    import torch
    with pytest.raises(TypeError):
        L.check_device_state(torch.zeros(16, dtype=torch.float64), 16)
    L.check_device_state(_FakeCudaTensor(16), 16, device=0)
    L.check_device_state(_FakeCudaTensor(16, itemsize=16, complex_=True), 16, complex_=True)
    with pytest.raises(ValueError):
        L.check_device_state(_FakeCudaTensor(15), 16)
    with pytest.raises(ValueError):
        L.check_device_state(_FakeCudaTensor(16, contiguous=False), 16)
    with pytest.raises(TypeError):
        L.check_device_state(_FakeCudaTensor(16, itemsize=4), 16)          # float32
    with pytest.raises(TypeError):
        L.check_device_state(_FakeCudaTensor(16, floating=False), 16)      # int64
    with pytest.raises(TypeError):
        L.check_device_state(_FakeCudaTensor(16), 16, complex_=True)       # real for complex
    with pytest.raises(ValueError):
        L.check_device_state(_FakeCudaTensor(16, index=1), 16, device=0)


def test_host_state_checks():
    L.check_host_state(np.zeros(12), 12)
    L.check_host_state(np.zeros((3, 4)), 12)
    L.check_host_state(np.zeros(12, dtype=np.complex128), 12, complex_=True)
    with pytest.raises(TypeError):
        L.check_host_state(np.zeros(12, dtype=np.float32), 12)
    with pytest.raises(TypeError):
        L.check_host_state([0.0] * 12, 12)
    with pytest.raises(ValueError):
        L.check_host_state(np.zeros(11), 12)
    with pytest.raises(ValueError):
        L.check_host_state(np.zeros((4, 6))[:, ::2], 12)
