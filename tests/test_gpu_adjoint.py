"""Per-cell wave speed and the discrete adjoint on the GPU, against the oracle."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import adjoint as oadj
from oracle import pipeline
from paper_2310_14712_gb300 import workloads

from parity_util import check_state

pytestmark = pytest.mark.gpu


def _case(nsrc=2, ncells=(8, 8), p=3, nsteps=60, seed=1):
    rng = np.random.default_rng(seed)
    nc = ncells[0] * ncells[1]
    xs = (np.arange(ncells[0]) + 0.5) / ncells[0]
    ys = (np.arange(ncells[1]) + 0.5) / ncells[1]
    X, Y = np.meshgrid(xs, ys)
    c = (1.0 + 0.15 * np.sin(2.1 * X + 0.7) * np.cos(1.7 * Y - 0.3)).ravel()
    w = workloads.Workload("adjcase", 2, (0.0, 0.0), (1.0, 1.0), ncells, p, 1e-5, 2,
                           np.array([[0.55, 0.5, 0.2, 0.2]]), rng.uniform(0.15, 0.35, (nsrc, 2)), 5.0, 0.06, 0)
    w.cell_c = c
    s = pipeline.setup(**dict(w.kwargs(), src_pos=w.src_pos[:1]))
    w.dt = s.dt   # one fixed step for every model below
    nn = s.grid.nnodes
    nx = ncells[0] * p + 1
    rec = np.arange(nn - nx, nn, 3, dtype=np.int64)[:8]       # top edge
    data = 1e-3 * rng.standard_normal((nsteps, nsrc, len(rec)))
    return w, c, rec, data, nsteps


def _oracle(w, c, rec, data, nsteps):
    J, g = 0.0, np.zeros(len(c))
    kw = dict(w.kwargs(), cell_c=c)
    pos = kw.pop("src_pos")
    for k in range(len(pos)):
        s = pipeline.setup(src_pos=pos[k:k + 1], **kw)
        Jk, gk = oadj.misfit_and_gradient(s, c, nsteps, rec, data[:, k, :])
        J += Jk
        g += gk
    return J, g


def test_per_cell_speed_forward_matches_oracle():
    from paper_2310_14712_gb300 import imex
    w, c, _, _, nsteps = _case(nsrc=1)
    with imex.Imex.from_workload(w) as g:
        g.step(nsteps)
        st = {k: g.fields(k, out=np.zeros(g.n_nodes)) for k in ("u", "u_prev_d", "v_c", "a_c")}
    s = pipeline.setup(**w.kwargs())
    ref = s.imex.run(nsteps)
    check_state(s, ref, st, w.holes, w.alpha, nsteps)


def test_adjoint_gradient_matches_oracle():
    from paper_2310_14712_gb300 import adjoint
    w, c, rec, data, nsteps = _case()
    J, g = adjoint.misfit_and_gradient(w, c, rec, data, nsteps, checkpoint_every=16)
    Jr, gr = _oracle(w, c, rec, data, nsteps)
    assert J == pytest.approx(Jr, rel=1e-10)
    assert np.linalg.norm(g - gr) <= 1e-8 * np.linalg.norm(gr)


def test_adjoint_checkpoint_interval_does_not_change_the_gradient():
    from paper_2310_14712_gb300 import adjoint
    w, c, rec, data, nsteps = _case(nsteps=30)
    ref = adjoint.misfit_and_gradient(w, c, rec, data, nsteps, checkpoint_every=30)
    for k in (1, 7):
        J, g = adjoint.misfit_and_gradient(w, c, rec, data, nsteps, checkpoint_every=k)
        assert J == ref[0] and np.array_equal(g, ref[1])


def test_adjoint_matches_central_differences_and_autograd():
    from paper_2310_14712_gb300 import adjoint
    w, c, rec, data, nsteps = _case(nsteps=40)
    ct = torch.tensor(c, dtype=torch.float64, requires_grad=True)
    J = adjoint.misfit(ct, w, rec, data, nsteps, 10, w.dt)
    (g,) = torch.autograd.grad(J, ct)
    J2, g2 = adjoint.misfit_and_gradient(w, c, rec, data, nsteps, 10, w.dt)
    assert float(J.detach()) == J2 and np.array_equal(g.numpy(), g2)

    def Jof(cc):
        tr = adjoint.traces(w, cc, rec, nsteps, w.dt)
        e = tr - data
        return 0.5 * float((e * e).sum())

    assert Jof(c) == pytest.approx(J2, rel=1e-12)
    for e in (9, 27, 45):
        h = 1e-6
        cp = c.copy(); cp[e] += h
        cm = c.copy(); cm[e] -= h
        fd = (Jof(cp) - Jof(cm)) / (2 * h)
        assert abs(fd - g2[e]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(g2).max()), (e, fd, g2[e])


def test_adjoint_full_size_against_central_differences():
    # 16 sources (columns), 64 receivers on the top edge, 2000 steps,
    # checkpoint every 100: two cells against central differences.
    from paper_2310_14712_gb300 import adjoint
    w = workloads.adjoint()
    rec = workloads.receiver_nodes(w, 64)
    c = np.asarray(w.cell_c, dtype=np.float64)
    dt = pipeline.setup(**dict(w.kwargs(), src_pos=w.src_pos[:1])).dt
    data = adjoint.traces(w, np.ones_like(c), rec, w.steps, dt)    # observed: homogeneous model
    J, g = adjoint.misfit_and_gradient(w, c, rec, data, w.steps, 100, dt)
    assert J > 0 and np.isfinite(g).all()

    def Jof(cc):
        e = adjoint.traces(w, cc, rec, w.steps, dt) - data
        return 0.5 * float((e * e).sum())

    for e in np.argsort(-np.abs(g))[:2]:
        h = 1e-6
        cp = c.copy(); cp[e] += h
        cm = c.copy(); cm[e] -= h
        fd = (Jof(cp) - Jof(cm)) / (2 * h)
        assert abs(fd - g[e]) <= 1e-4 * abs(fd), (e, fd, g[e])


def test_adjoint_3d_matches_oracle():
    # 4 x 3 x 3 cells, p = 2, one void, per-cell speed, 2 sources, 25 steps.
    from paper_2310_14712_gb300 import adjoint
    rng = np.random.default_rng(3)
    w = workloads.Workload("adj3", 3, (0.0, 0.0, 0.0), (1.0, 0.8, 0.6), (4, 3, 3), 2, 1e-4, 2,
                           np.array([[0.55, 0.4, 0.3, 0.22, 0.18, 0.15]]),
                           np.array([[0.2, 0.25, 0.2], [0.8, 0.55, 0.35]]), 3.0, 0.1, 0)
    c = 1.0 + 0.1 * rng.standard_normal(4 * 3 * 3)
    w.cell_c = c
    s = pipeline.setup(**dict(w.kwargs(), src_pos=w.src_pos[:1]))
    w.dt = s.dt
    nn = s.grid.nnodes
    rec = np.arange(nn - 12, nn, 2, dtype=np.int64)
    nsteps = 25
    data = 1e-3 * rng.standard_normal((nsteps, 2, len(rec)))
    J, g = adjoint.misfit_and_gradient(w, c, rec, data, nsteps, checkpoint_every=7)
    Jr, gr = _oracle(w, c, rec, data, nsteps)
    assert J == pytest.approx(Jr, rel=1e-10)
    assert np.linalg.norm(g - gr) <= 1e-8 * np.linalg.norm(gr)
