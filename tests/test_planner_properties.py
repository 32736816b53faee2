"""Property tests of the host planner (no device): random decompositions against the oracle."""
import numpy as np
import pytest

from oracle import decompose
from paper_1505_02248_gb300 import build as B
from paper_1505_02248_gb300 import lem as L

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


@st.composite
def _plans(draw):
    nd = draw(st.integers(1, 2))
    shape = tuple(draw(st.integers(1, 60)) for _ in range(nd))
    bc = tuple(draw(st.sampled_from(["dirichlet", "periodic"])) for _ in range(nd))
    tile = tuple(draw(st.integers(1, max(1, s))) for s in shape)
    H = tuple(draw(st.integers(0, 12)) for _ in range(nd))
    return shape, bc, tile, H


@settings(max_examples=150, deadline=None)
@given(_plans())
def test_planner_matches_oracle_on_random_plans(lib, plan):
    """Random meshes, tiles, overlaps and boundary conditions (ragged tiles, windows clipped at
    walls or wrapped, whole-axis periodic windows): every tile's owner and window node sets and
    the owner positions inside the window match the oracle's decomposition (Sec. 3, Fig. 3)."""
    shape, bc, tile, H = plan
    coef = {k: 1.0 for k in "CWESN"}
    q = L.plan_query(shape, bc, coef, 1.0, tile, H)
    wins = decompose(shape, bc, tile, H)
    assert q["ntiles"] == len(wins)
    nx = shape[-1]
    ny = shape[0] if len(shape) == 2 else 1
    for i, w in enumerate(wins):
        oy, ox, wy, wx, iy, ix, ey, ex, ty, tx = (int(v) for v in q["tiles"][i][:10])
        M = np.array([((oy + a) % ny) * nx + (ox + b) % nx for a in range(wy) for b in range(wx)])
        D = np.array([(ty + a) * nx + tx + b for a in range(ey) for b in range(ex)])
        assert np.array_equal(M, w.M) and np.array_equal(D, w.D)
        assert np.array_equal(np.array([(iy + a) * wx + ix + b for a in range(ey) for b in range(ex)]), w.d_pos)
    # every node has exactly one owner
    owners = np.concatenate([w.D for w in wins])
    assert np.array_equal(np.sort(owners), np.arange(int(np.prod(shape))))
