"""Seeded synthetic workloads: geometry, sources and material inputs.

This module only draws random numbers and fixes constants; it contains none of
the method's arithmetic.  It is the single source of inputs for both the CUDA
path and the CPU checker, so that both see identical holes, sources and wave
speeds.  It imports nothing from the rest of the package.

Workloads (the paper's perforated plate and voided solid stand in for the
paper's unpublished random holes and STL pillar):
  plate16      [0,1]^2 minus one centred circle r=0.2; 16x16 cells, p=4,
               alpha=1e-5, quadtree depth 3; Ricker f0=5 at (0.2,0.2); 500 steps
  plate256     [0,2]x[0,1] minus 24 seeded non-overlapping circles r~U[0.03,0.08],
               centres x~U[0.4,2], y~U[0,1]; 256x128 cells, p=4, alpha=1e-5,
               depth 3; Ricker f0=20 at (0.1,0.5); 5000 steps
  multisource  plate16 geometry, 64 seeded source positions inside the physical
               domain, Ricker f0=20; 2000 steps
  voids3d      [0,1]x[0,1]x[0,0.5] minus 40 seeded axis-aligned ellipsoids,
               semi-axes U[0.03,0.1]; 64x64x32 cells, p=3, octree depth 2; 1000 steps
  adjoint      plate16 geometry with a smooth seeded per-cell wave speed in
               [0.8,1.2], 16 sources, 64 receivers on the top edge; 2000 steps
Spatial source: Gaussian bell of amplitude 10 (the paper's bell) with width
sigma = 0.12 c / f0 (the paper's ratio of bell width to dominant wavelength).
"""
from dataclasses import dataclass, field
from typing import Optional
import numpy as np

RICKER, GAUSS_DERIV, SINE_BURST = 0, 1, 2


@dataclass
class Workload:
    name: str
    dim: int
    lo: tuple
    hi: tuple
    ncells: tuple
    p: int
    alpha: float
    depth: int
    holes: np.ndarray                 # (nholes, 2*dim): centre, semi-axes
    src_pos: np.ndarray               # (nsrc, dim)
    f0: float
    src_sigma: float
    steps: int
    src_amp: float = 10.0
    wavelet: int = RICKER
    rho: float = 1.0
    c0: float = 1.0
    cell_c: Optional[np.ndarray] = None   # per-cell wave speed, flat order x fastest
    receivers: Optional[np.ndarray] = None
    dt: float = 0.0                   # <= 0: 0.9 x uncut-cell critical step
    extra: dict = field(default_factory=dict)

    def kwargs(self):
        """Plain arguments for a discretisation (geometry, order, source, material)."""
        return dict(dim=self.dim, lo=self.lo, hi=self.hi, ncells=self.ncells, p=self.p,
                    alpha=self.alpha, depth=self.depth, holes=self.holes,
                    src_pos=self.src_pos, f0=self.f0, src_sigma=self.src_sigma,
                    src_amp=self.src_amp, wavelet=self.wavelet, rho=self.rho,
                    c0=self.c0, cell_c=self.cell_c, dt=self.dt)

    def grid_nodes(self):
        return int(np.prod([n * self.p + 1 for n in self.ncells]))


def _non_overlapping(rng, n, centre_lo, centre_hi, axis_lo, axis_hi, dim, equal_axes):
    holes = []
    tries = 0
    while len(holes) < n:
        tries += 1
        if tries > 100000:
            raise RuntimeError("hole sampling did not converge")
        c = rng.uniform(centre_lo, centre_hi)
        if equal_axes:
            a = np.full(dim, rng.uniform(axis_lo, axis_hi))
        else:
            a = rng.uniform(axis_lo, axis_hi, size=dim)
        ok = True
        for h in holes:
            if np.linalg.norm(c - h[:dim]) <= a.max() + h[dim:].max():
                ok = False
                break
        if ok:
            holes.append(np.concatenate([c, a]))
    return np.asarray(holes)


def plate16(steps=500):
    return Workload("plate16", 2, (0.0, 0.0), (1.0, 1.0), (16, 16), 4, 1e-5, 3,
                    np.array([[0.5, 0.5, 0.2, 0.2]]), np.array([[0.2, 0.2]]),
                    5.0, 0.12 / 5.0, steps)


def plate256(steps=5000, seed=2):
    rng = np.random.default_rng(seed)
    holes = _non_overlapping(rng, 24, np.array([0.4, 0.0]), np.array([2.0, 1.0]),
                             0.03, 0.08, 2, True)
    return Workload("plate256", 2, (0.0, 0.0), (2.0, 1.0), (256, 128), 4, 1e-5, 3,
                    holes, np.array([[0.1, 0.5]]), 20.0, 0.12 / 20.0, steps)


def _inside_points(rng, n, lo, hi, holes, dim, margin=0.0):
    pts = []
    while len(pts) < n:
        x = rng.uniform(np.asarray(lo) + margin, np.asarray(hi) - margin)
        ok = True
        for h in holes:
            if (((x - h[:dim]) / h[dim:]) ** 2).sum() <= 1.0:
                ok = False
                break
        if ok:
            pts.append(x)
    return np.asarray(pts)


def multisource(nsrc=64, steps=2000, seed=3):
    w = plate16(steps)
    rng = np.random.default_rng(seed)
    w.name = "multisource"
    w.src_pos = _inside_points(rng, nsrc, w.lo, w.hi, w.holes, 2)
    w.f0 = 20.0
    w.src_sigma = 0.12 / 20.0
    return w


def voids3d(steps=1000, seed=4, ncells=(64, 64, 32)):
    rng = np.random.default_rng(seed)
    holes = _non_overlapping(rng, 40, np.array([0.0, 0.0, 0.0]), np.array([1.0, 1.0, 0.5]),
                             0.03, 0.1, 3, False)
    return Workload("voids3d", 3, (0.0, 0.0, 0.0), (1.0, 1.0, 0.5), tuple(ncells), 3, 1e-5, 2,
                    holes, np.array([[0.1, 0.5, 0.25]]), 20.0, 0.12 / 20.0, steps)


def adjoint(nsrc=16, nrec=64, steps=2000, seed=5):
    w = plate16(steps)
    rng = np.random.default_rng(seed)
    w.name = "adjoint"
    nx, ny = w.ncells
    xs = (np.arange(nx) + 0.5) / nx
    ys = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    field_ = np.zeros_like(X)
    for _ in range(4):
        kx, ky = rng.integers(1, 4, size=2)
        ph = rng.uniform(0, 2 * np.pi, size=2)
        field_ += np.cos(np.pi * kx * X + ph[0]) * np.cos(np.pi * ky * Y + ph[1])
    field_ = field_ / np.abs(field_).max()
    w.cell_c = (1.0 + 0.2 * field_).ravel()      # flat order, x fastest
    w.src_pos = _inside_points(rng, nsrc, w.lo, w.hi, w.holes, 2, margin=0.05)
    w.receivers = np.stack([np.linspace(0.05, 0.95, nrec), np.full(nrec, 0.98)], axis=1)
    return w


WORKLOADS = {"plate16": plate16, "plate256": plate256, "multisource": multisource,
             "voids3d": voids3d, "adjoint": adjoint}


def get(name, **kw):
    return WORKLOADS[name](**kw)


def source_signature(n, dt, seed=7, fmax=20.0, ncomp=8):
    """A seeded, smooth source signature of n samples at spacing dt: a sum of
    `ncomp` sinusoids with random frequencies in [0.1, 1] fmax, amplitudes and
    phases, under a raised-cosine window.  Input data for the user-supplied
    source-samples path (a stand-in for a recorded or inverted signature)."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.1, 1.0, ncomp) * fmax
    a = rng.uniform(0.5, 1.0, ncomp)
    ph = rng.uniform(0.0, 2.0 * np.pi, ncomp)
    t = np.arange(n) * dt
    sig = (a[None, :] * np.sin(2.0 * np.pi * f[None, :] * t[:, None] + ph[None, :])).sum(axis=1)
    window = 0.5 - 0.5 * np.cos(2.0 * np.pi * np.arange(n) / max(n - 1, 1))
    return np.ascontiguousarray(sig * window)


def receiver_nodes(w, nrec):
    """Canonical node ids of `nrec` receivers evenly spaced along the top edge."""
    nx = w.ncells[0] * w.p + 1
    ny = w.ncells[1] * w.p + 1
    xs = np.linspace(0, nx - 1, nrec).round().astype(np.int64)
    return np.ascontiguousarray((ny - 1) * nx + xs, dtype=np.int64)
