"""Pins of the PSO oracle (Sec. III) and of its counter-based generator (CPU only)."""

import math
import os

import numpy as np

from oracle import pso_oracle as po

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = po.philox4x32_10(np.array(v[:4], dtype=np.uint64), np.array(v[4:6], dtype=np.uint64))
        assert [int(o) for o in out] == v[6:]


def test_uniforms_are_uniform_and_streams_independent():
    u = po.uniforms(3, 17, np.arange(50000), 0, seed=12345)
    w = po.uniforms(3, 17, np.arange(50000), 1, seed=12345)
    assert u.min() > 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.003 and abs(u.var() - 1 / 12) < 0.002
    assert abs(np.corrcoef(u[:, 0], w[:, 0])[0, 1]) < 0.02
    assert abs(np.corrcoef(u[:, 0], u[:, 1])[0, 1]) < 0.02


def test_one_step_by_hand(monkeypatch):
    """w = 0.9 at iteration 0, v = 0.1, x = 0.5, pbest = 0.7, lbest = 0.4, r1 = 1/4, r2 = 3/4:
    v' = 0.09 + 2 (1/4)(0.2) + 2 (3/4)(-0.1) = 0.04, x' = 0.54; a velocity beyond vmax is clamped."""
    cfg = po.PsoConfig(n_runs=1, n_particles=3, n_iter=10, vmax=0.5)
    s = po.PsoState(cfg)
    s.x[0] = 0.5
    s.v[0] = 0.1
    s.pbest_x[0] = 0.7
    s.pbest_f[0] = [10.0, 1.0, 1.0]      # particle 0's personal best is its own and stays
    s.pbest_x[0, 0] = 0.7
    s.pbest_x[0, 1:] = 0.4               # particles 1, 2: their lbest is particle 0's pbest (0.7)
    vals = {0: 0.25, 1: 0.75}
    monkeypatch.setattr(po, "uniforms", lambda run, it, p, stream, seed: np.full((len(p), 4), vals[stream]))
    po.update(cfg, s, 0, np.array([[0.0, 0.0, 0.0]]), np.zeros((1, 3), dtype=np.int64))
    # particle 0: pbest 0.7, lbest 0.7 (itself) -> 0.09 + 0.1 + 0.3 = 0.49
    np.testing.assert_allclose(s.v[0, 0], 0.09 + 2 * 0.25 * 0.2 + 2 * 0.75 * 0.2, rtol=1e-15)
    # particle 1: pbest 0.4, lbest 0.7 -> 0.09 + 2 (1/4)(-0.1) + 2 (3/4)(0.2) = 0.34
    np.testing.assert_allclose(s.v[0, 1], 0.09 - 0.05 + 0.3, rtol=1e-14)
    np.testing.assert_allclose(s.x[0, 1], 0.5 + 0.34, rtol=1e-14)
    s.x[0] = 0.0
    s.v[0] = 0.4
    po.update(cfg, s, 1, np.array([[0.0, 0.0, 0.0]]), np.zeros((1, 3), dtype=np.int64))
    assert np.all(s.v[0] == 0.5)         # clamped at vmax


def test_ring_local_best():
    cfg = po.PsoConfig(n_runs=1, n_particles=4, n_neighbours=1)
    lb = po.local_best(cfg, np.array([[5.0, 1.0, 7.0, 3.0]]))
    assert list(lb[0]) == [0, 2, 2, 2]
    lb = po.local_best(cfg, np.array([[2.0, 2.0, 1.0, 2.0]]))   # ties: lowest index
    assert list(lb[0]) == [0, 0, 1, 0]


def test_particles_outside_the_box_are_not_evaluated():
    cfg = po.PsoConfig(n_runs=1, n_particles=2)
    s = po.init_state(cfg)
    s.x[0, 1, 2] = 1.5
    po.update(cfg, s, 0, np.array([[3.0, 99.0]]), np.array([[7, 8]]))
    assert s.pbest_f[0, 0] == 3.0 and s.pbest_f[0, 1] == -np.inf and s.pbest_tc[0, 1] == -1


def test_search_finds_the_maximum_of_a_smooth_function():
    """Best-of-M lbest PSO locates the unique maximum of a smooth function inside the box."""
    cfg = po.PsoConfig(n_runs=2, n_particles=20, n_iter=200, seed=7,
                       box=(0.0, 2 * math.pi, -0.5 * math.pi, 0.5 * math.pi, 1.0, 2.0, 0.1, 0.2))
    target = np.array([2.0, 0.3, 1.3, 0.17])
    scale = np.array([2 * math.pi, math.pi, 1.0, 0.1])

    def fit(theta):
        d = (theta - target) / scale
        return 100.0 - np.sum(d * d, axis=1), np.arange(len(theta))

    res, s = po.run_search(cfg, fit)
    best = max(res, key=lambda r: r[0])
    np.testing.assert_allclose(best[1], target, atol=1e-3 * scale.max())
    assert np.all(np.diff(np.sort(s.pbest_f.ravel())) >= 0)


def test_search_is_reproducible_from_the_seed():
    cfg = po.PsoConfig(n_runs=2, n_particles=8, n_iter=20, seed=3)
    f = lambda th: (np.cos(th[:, 0]) + th[:, 2], np.zeros(len(th), dtype=np.int64))
    a, _ = po.run_search(cfg, f)
    b, _ = po.run_search(cfg, f)
    cfg.seed = 4
    c, _ = po.run_search(cfg, f)
    assert [r[0] for r in a] == [r[0] for r in b]
    assert [r[0] for r in a] != [r[0] for r in c]
