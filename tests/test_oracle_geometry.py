"""Pins of the oracle's geometry (Sec. Spatial discretization, FCM) against brute force."""
import numpy as np

from oracle import geometry as G


def _brute(holes, lo, hi, n=61):
    xs = np.linspace(lo[0], hi[0], n)
    ys = np.linspace(lo[1], hi[1], n)
    X, Y = np.meshgrid(xs, ys)
    phys = holes.physical(np.stack([X.ravel(), Y.ravel()], axis=1))
    return phys.any(), (~phys).any()


def test_classify_matches_sampling():
    rng = np.random.default_rng(0)
    checked = 0
    for _ in range(400):
        c = rng.uniform(0, 1, 2)
        a = rng.uniform(0.05, 0.4, 2)
        holes = G.Holes(np.concatenate([c, a])[None], 2)
        lo = rng.uniform(0, 1, 2)
        hi = lo + rng.uniform(0.02, 0.3, 2)
        t = holes.classify_box(lo, hi)
        has_phys, has_fict = _brute(holes, lo, hi)
        if t == G.EMPTY:
            assert not has_phys
        elif t == G.UNCUT:
            assert not has_fict
        else:
            # sampling may miss a thin sliver; accept only if a finer sampling agrees
            if not (has_phys and has_fict):
                hp, hf = _brute(holes, lo, hi, n=801)
                assert hp and hf
        checked += 1
    assert checked == 400


def test_tangent_box_is_uncut():
    holes = G.Holes(np.array([[0.0, 0.0, 1.0, 1.0]]), 2)
    assert holes.classify_box(np.array([1.0, -0.5]), np.array([2.0, 0.5])) == G.UNCUT
    assert holes.classify_box(np.array([0.5, -0.5]), np.array([2.0, 0.5])) == G.CUT
    assert holes.classify_box(np.array([-0.5, -0.5]), np.array([0.5, 0.5])) == G.EMPTY


def test_ellipsoid_3d_classification():
    holes = G.Holes(np.array([[0.5, 0.5, 0.5, 0.3, 0.2, 0.1]]), 3)
    assert holes.classify_box(np.array([0.45, 0.45, 0.45]), np.array([0.55, 0.55, 0.55])) == G.EMPTY
    assert holes.classify_box(np.array([0.75, 0.45, 0.45]), np.array([0.85, 0.55, 0.55])) == G.CUT
    assert holes.classify_box(np.array([0.45, 0.45, 0.61]), np.array([0.55, 0.55, 0.7])) == G.UNCUT
