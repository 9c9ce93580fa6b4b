"""Pins of the oracle's gradient of Gamma^2 at fixed t_c (CPU only)."""

import numpy as np
import pytest

import synthdata as sd
from oracle import fcas_oracle as o


@pytest.fixture(scope="module")
def setup():
    w = sd.SMALL
    data = sd.make_dataset(w, 2)
    return o.OracleSetup(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high)


def test_single_t_statistic_equals_the_fft_curve(setup):
    for th in sd.make_particles(sd.SMALL, 3, seed=2):
        curve = o.fitness_curve(setup, th)
        for t in (0, 17, int(np.argmax(curve)), setup.n_fft - 1):
            assert o.statistic_at(setup, th, t) == pytest.approx(curve[t], rel=1e-10, abs=1e-12 * curve.max())


@pytest.mark.parametrize("rel_step", [1e-6, 1e-5, 1e-4, 1e-3])
def test_complex_step_gradient_matches_central_differences(setup, rel_step):
    """Central differences converge to the complex-step gradient at second order: relative error
    <= 1e-7 + C h^2 (h the relative step; C covers the third derivative of the chirp phase)."""
    th = sd.make_particles(sd.SMALL, 1, seed=9)[0]
    t = int(np.argmax(o.fitness_curve(setup, th)))
    g = o.gradient(setup, th, t)
    scale = np.array([1.0, 1.0, th[2], th[3]])
    for j in range(4):
        h = rel_step * scale[j]
        e = np.zeros(4)
        e[j] = h
        fd = (o.statistic_at(setup, th + e, t) - o.statistic_at(setup, th - e, t)) / (2 * h)
        assert abs(fd - g[j]) <= (1e-7 + 5e4 * rel_step ** 2) * abs(g[j]), (j, fd, g[j])


def test_central_differences_converge_at_second_order(setup):
    th = sd.make_particles(sd.SMALL, 1, seed=9)[0]
    t = int(np.argmax(o.fitness_curve(setup, th)))
    g = o.gradient(setup, th, t)
    e = np.array([0.0, 0.0, 1.0, 0.0])

    def err(rs):
        h = rs * th[2]
        return abs((o.statistic_at(setup, th + h * e, t) - o.statistic_at(setup, th - h * e, t)) / (2 * h) - g[2])

    assert err(1e-3) / err(1e-4) > 50.0            # h^2 scaling toward the complex-step value
