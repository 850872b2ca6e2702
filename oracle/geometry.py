"""Immersed geometry of the finite/spectral cell method (oracle, test infrastructure).

Sec. "Spatial discretization": the physical domain Omega_p is embedded in a
box Omega meshed by a Cartesian grid; the indicator alpha(x) is 1 in Omega_p
and alpha_f = 10^-beta in the fictitious part Omega_f.  Here Omega_p is the
box minus a set of axis-aligned ellipses/ellipsoids ("holes"; circles when the
semi-axes are equal), as in the perforated-plate and void examples.

Readings of the paper taken here:
  * a point is physical iff it lies strictly outside every hole,
    sum(((x - c) / a)^2) > 1;
  * a (sub)cell is *cut* iff the boundary of some hole meets its interior; a
    cell that only touches a hole boundary at an edge or corner is uncut;
  * a cell lying inside one closed hole is *empty* and is discarded
    (Sec. 2D example: "discard finite cells that are entirely outside the
    physical domain").

The box test is exact for axis-aligned ellipsoids: after scaling space by the
semi-axes the hole is the unit ball, and the nearest and farthest points of the
scaled box from the centre decide inside / outside / crossing.

Pins: tests/test_oracle_geometry.py (brute-force sampling of boxes against the
exact classification; fill-ratio of a circle cut converging to the analytic area).
"""
import numpy as np

UNCUT, CUT, EMPTY = 0, 1, 2


class Holes:
    """Axis-aligned ellipsoidal holes: rows (centre[dim], semi_axes[dim])."""

    def __init__(self, holes, dim):
        holes = np.asarray(holes, dtype=np.float64).reshape(-1, 2 * dim)
        self.dim = dim
        self.c = holes[:, :dim]
        self.a = holes[:, dim:]

    def physical(self, x):
        """Boolean mask: points x (n, dim) strictly outside every hole."""
        x = np.atleast_2d(x)
        inside = np.zeros(len(x), dtype=bool)
        for c, a in zip(self.c, self.a):
            inside |= (((x - c) / a) ** 2).sum(axis=1) <= 1.0
        return ~inside

    def classify_box(self, lo, hi):
        """UNCUT, CUT or EMPTY for the closed box [lo, hi] (exact test)."""
        lo = np.asarray(lo, dtype=np.float64)
        hi = np.asarray(hi, dtype=np.float64)
        cut = False
        for c, a in zip(self.c, self.a):
            slo = (lo - c) / a
            shi = (hi - c) / a
            near = np.clip(0.0, slo, shi)                  # nearest point to the centre
            far = np.maximum(np.abs(slo), np.abs(shi))     # farthest corner
            dmin2 = float((near ** 2).sum())
            dmax2 = float((far ** 2).sum())
            if dmax2 <= 1.0:
                return EMPTY
            if dmin2 < 1.0:
                cut = True
        return CUT if cut else UNCUT


class HalfSpace:
    """Physical domain {x : x[axis] < level}; used for the paper's single-cut-cell study
    (Sec. "Motivation", Fig. fillRatio: a cell cut by a horizontal boundary)."""

    def __init__(self, axis, level, dim):
        self.axis, self.level, self.dim = axis, level, dim

    def physical(self, x):
        x = np.atleast_2d(x)
        return x[:, self.axis] < self.level

    def classify_box(self, lo, hi):
        if hi[self.axis] <= self.level:
            return UNCUT
        if lo[self.axis] >= self.level:
            return EMPTY
        return CUT
