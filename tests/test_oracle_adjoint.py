"""Pins of the discrete adjoint (oracle/adjoint.py): central finite
differences of the misfit, on small problems with and without cut cells."""
import numpy as np
import pytest

from oracle import adjoint, pipeline
from paper_2310_14712_gb300 import workloads


def _case(holes, ncells=(6, 6), nsteps=40, seed=0):
    w = workloads.Workload("adj", 2, (0.0, 0.0), (1.0, 1.0), ncells, 2, 1e-5, 2,
                           np.asarray(holes, dtype=float).reshape(-1, 4),
                           np.array([[0.3, 0.35]]), 4.0, 0.1, 0)
    rng = np.random.default_rng(seed)
    nc = ncells[0] * ncells[1]
    c = 1.0 + 0.15 * rng.standard_normal(nc).clip(-1.3, 1.3)
    kw = w.kwargs()
    kw["cell_c"] = c
    kw["dt"] = 0.0
    # one fixed step for every speed model (the critical step of the fastest uncut cell
    # of the reference model, times 0.8)
    s0 = pipeline.setup(**kw)
    kw["dt"] = 0.8 / 0.9 * s0.dt
    rec = np.array([s0.grid.nnodes - 1 - 2 * k for k in range(5)])
    data = np.zeros((nsteps, len(rec)))
    return kw, c, rec, data, nsteps


def _J(kw, c, rec, data, nsteps):
    kw = dict(kw)
    kw["cell_c"] = c
    return adjoint.forward_misfit(pipeline.setup(**kw), nsteps, rec, data)


@pytest.mark.parametrize("holes", [np.zeros((0, 4)), [[0.55, 0.6, 0.23, 0.23]]])
def test_adjoint_gradient_matches_central_differences(holes):
    kw, c, rec, data, nsteps = _case(holes)
    s = pipeline.setup(**dict(kw, cell_c=c))
    J, g = adjoint.misfit_and_gradient(s, c, nsteps, rec, data)
    assert J == pytest.approx(_J(kw, c, rec, data, nsteps), rel=1e-12)
    rng = np.random.default_rng(5)
    cells = np.flatnonzero(s.disc.cell_type != 2)
    for e in rng.choice(cells, 6, replace=False):
        h = 1e-6
        cp = c.copy(); cp[e] += h
        cm = c.copy(); cm[e] -= h
        fd = (_J(kw, cp, rec, data, nsteps) - _J(kw, cm, rec, data, nsteps)) / (2 * h)
        assert abs(fd - g[e]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(g).max()), (e, fd, g[e])
