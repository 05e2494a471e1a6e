"""Pins of the oracle's recursive re-meshing (Sec. 4.1) on the CPU."""
import numpy as np

import oracle as O


def _cloud(n=3000, seed=1):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(n, 3))


def test_variation_formula():
    assert O.box_variation(np.array([1.0, 3.0, 2.0])) == 2.0 * (2.0 / 4.0)
    assert O.box_variation(np.array([5.0, 5.0])) == 0.0


def test_constant_tracer_is_one_box_plus_boundary():
    p = _cloud()
    pts, flags, leaves = O.remesh(p, np.full(len(p), 7.0), 0.4, 12, 4)
    assert len(leaves) == 1 and flags.sum() == 6 * 16 - 12 * 4 + 8       # 56 surface nodes of a 4^3 lattice
    assert np.allclose(pts[0], (p.min(axis=0) + p.max(axis=0)) / 2)
    b = pts[flags == 1]
    lo, hi = p.min(axis=0), p.max(axis=0)
    assert np.all(np.any(np.isclose(b, lo) | np.isclose(b, hi), axis=1))   # every boundary node on a face


def test_leaves_partition_the_points_and_meet_the_criterion():
    p = _cloud(4000, 2)
    rho = 1e3 * np.exp(-3 * np.linalg.norm(p, axis=1)) + 1.0
    r_max, lmax = 0.3, 6
    _, _, leaves = O.remesh(p, rho, r_max, lmax, 3)
    seen = np.concatenate([idx for _, _, _, idx in leaves])
    assert np.array_equal(np.sort(seen), np.arange(len(p)))             # every point in exactly one leaf
    for lo, hi, level, idx in leaves:
        assert level == lmax or O.box_variation(rho[idx]) <= r_max
        q = p[idx]
        assert np.array_equal(lo, q.min(axis=0)) and np.array_equal(hi, q.max(axis=0))   # cropped


def test_step_tracer_refines_only_at_the_step():
    # rho jumps across the plane x = 0.05: only boxes straddling it divide, down to the last level
    p = _cloud(6000, 3)
    rho = np.where(p[:, 0] < 0.05, 1.0, 10.0)
    _, _, leaves = O.remesh(p, rho, 0.5, 5, 2)
    for lo, hi, level, idx in leaves:
        straddles = rho[idx].min() != rho[idx].max()
        assert straddles == (level == 5) or not straddles
        if level < 5:
            assert not straddles
    assert max(l for _, _, l, _ in leaves) == 5
    # far from the step the boxes stay coarse
    assert min(l for _, _, l, _ in leaves) <= 2
