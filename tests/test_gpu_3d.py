"""3D path (tensor-grid explicit apply with three passes, octree cut cells,
the same implicit solve) against the oracle."""
import numpy as np
import pytest

from oracle import pipeline
from paper_2310_14712_gb300 import workloads

from parity_util import check_state

pytestmark = pytest.mark.gpu


def _imex():
    from paper_2310_14712_gb300 import imex
    return imex


def _box3(ncells, p, holes, hi=(1.0, 0.8, 0.6), depth=2):
    return workloads.Workload("box3", 3, (0.0, 0.0, 0.0), hi, tuple(ncells), p, 1e-5, depth,
                              np.asarray(holes, dtype=float).reshape(-1, 6),
                              np.array([[0.31, 0.27, 0.22]]), 3.0, 0.1, 0)


def _run(w, nsteps):
    imex = _imex()
    with imex.Imex.from_workload(w) as g:
        g.step(nsteps)
        st = {k: g.fields(k, out=np.zeros(g.n_nodes)) for k in ("u", "u_prev_d", "v_c", "a_c")}
        info = g.info()
    return st, info


def _check(w, nsteps):
    st, info = _run(w, nsteps)
    s = pipeline.setup(**w.kwargs())
    ref = s.imex.run(nsteps)
    e_phys, e_all = check_state(s, ref, st, w.holes, w.alpha, nsteps)
    return e_phys, e_all, info


def test_3d_box_without_voids():
    # Every DOF explicit: the three-pass apply alone.
    _, _, info = _check(_box3((5, 3, 4), 3, np.zeros((0, 6))), 30)
    assert info["n_c"] == 0


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_3d_orders_ragged_grid_with_a_void(p):
    # 5 x 3 x 4 cells (no tile multiple), one ellipsoidal void crossing a face.
    w = _box3((5, 3, 4), p, [[0.55, 0.75, 0.3, 0.22, 0.17, 0.2]])
    _, _, info = _check(w, 25)
    assert info["n_c"] > 0 and info["n_d"] > 0


def test_3d_seeded_voids():
    w = workloads.voids3d(ncells=(6, 6, 3))
    w.holes = w.holes[:6]
    _check(w, 40)


def test_3d_tile_sizes_agree_bitwise(monkeypatch):
    out = {}
    w = _box3((5, 4, 3), 3, [[0.5, 0.4, 0.3, 0.2, 0.2, 0.15]])
    for tile in ("large", "small"):
        monkeypatch.setenv("IMEX_EXPLICIT_TILE", tile)
        st, info = _run(w, 20)
        out[tile] = (st["u"], info["explicit_tile_cells"])
    assert out["large"][1] != out["small"][1]
    assert np.array_equal(out["large"][0], out["small"][0])
