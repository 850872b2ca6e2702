"""One workload end to end on the CPU (oracle, test infrastructure).

Puts together: discretisation and partition (Sec. Spatial discretization,
Sec. Partitioning), the time step rule, and the Newmark IMEX loop
(Fig. TrapCDMIMEX).  The caller passes plain data (box, cells, order, holes,
sources ...); nothing here imports the CUDA package.

Time step rule (reading pinned by Table criticaltimestepsizes): when dt <= 0
the step is 0.9 times the cell-wise critical step of an uncut cell,
2 / sqrt(lambda_max(K_e, M_e)), for the largest wave speed among uncut cells.

Multiple sources are independent right-hand sides: each is run as its own
simulation (plain loop), which is what the batched GPU form must reproduce
column by column.

Pins (tests/test_oracle_pipeline.py): the time-step rule under wave-speed
scaling (speed 2 halves dt exactly; the fastest uncut cell decides, cut
cells do not); the source columns adding up to the run with all sources.
"""
import numpy as np

from .discretize import Grid, discretize, uncut_critical_dt, UNCUT
from .geometry import Holes
from .integrators import NewmarkImex
from . import sources


class Setup:
    pass


def setup(dim, lo, hi, ncells, p, alpha, depth, holes, src_pos, f0,
          src_sigma, src_amp=10.0, wavelet=sources.RICKER, rho=1.0, c0=1.0,
          cell_c=None, dt=0.0, dt_factor=0.9, geom=None, quad_reverse=False):
    """Discretise one workload and build its IMEX integrator (one source column).

    quad_reverse: sum every element quadrature in reverse point order (the
    same system up to roundoff; see discretize).  The arguments are kept as
    Setup.args so that the same workload can be set up again."""
    args = dict(dim=dim, lo=lo, hi=hi, ncells=ncells, p=p, alpha=alpha, depth=depth, holes=holes,
                src_pos=src_pos, f0=f0, src_sigma=src_sigma, src_amp=src_amp, wavelet=wavelet,
                rho=rho, c0=c0, cell_c=cell_c, dt=dt, dt_factor=dt_factor, geom=geom)
    grid = Grid(lo, hi, ncells, p)
    geom = Holes(holes, dim) if geom is None else geom
    fx = sources.bell(src_pos, src_sigma, src_amp)
    disc = discretize(grid, geom, alpha, depth, rho, c0, cell_c, fx, quad_reverse)
    if dt <= 0:
        if cell_c is None:
            cmax = c0
        else:
            cmax = float(np.max(np.asarray(cell_c)[disc.cell_type == UNCUT]))
        dt = dt_factor * uncut_critical_dt(p, grid.h, rho, cmax)
    ft = sources.wavelet(wavelet, f0)
    s = Setup()
    s.grid, s.disc, s.dt, s.ft, s.geom = grid, disc, dt, ft, geom
    s.args = args
    s.imex = NewmarkImex(disc.M, disc.K, disc.fx, ft, dt, disc.is_c, disc.is_d)
    return s


def setup_columns(src_pos, **kw):
    """Independent source columns: one single-source setup per position.

    Column k is the whole method run with the bell at src_pos[k] alone; the
    columns share nothing but the inputs (a plain loop, no batching)."""
    pos = np.asarray(src_pos, dtype=np.float64)
    return [setup(src_pos=pos[k:k + 1], **kw) for k in range(len(pos))]


def run(s, nsteps, u0=None, v0=None, callback=None):
    """Run `nsteps` IMEX steps from the initial state; returns the ImexState."""
    return s.imex.run(nsteps, u0=u0, v0=v0, callback=callback)


def relative_l2(a, b, mask=None):
    """||a - b|| / ||b|| over `mask` (all entries when None)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if mask is not None:
        a, b = a[mask], b[mask]
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))
