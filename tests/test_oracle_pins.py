"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics (CPU only).

Each pin is chosen so that a plausible mistake in the oracle (a dropped term, a sign, an index,
a normalisation factor, a transposed operand) fails at least one of them; the planted-mistake
tests at the end check that explicitly.
"""

import dataclasses
import math
import os

import numpy as np
import pytest

import synthdata as sd
from oracle import fcas_oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _setup(w, data):
    return o.OracleSetup(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high)


def _truth(w, inj):
    t0, _, t15, _ = o.chirp_times_from_masses(inj["m1"], inj["m2"], w.f_low)
    return [inj["alpha"], inj["delta"], t0, t15]


EXACT = dataclasses.replace(sd.SMALL, n_samples=sd.SMALL.n_fft)


# ---------------------------------------------------------------- chirp times (Sec. II.B, Sec. V)

def test_worked_example_duration_and_box():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "dns_chirp_duration.txt")) if l.strip() and l[0] != "#"]
    m1, m2, fstar, dur_min, t0lo, t0hi, t15lo, t15hi = (float(v) for v in rows[0])
    tau0, tau1, tau15, tau2 = o.chirp_times_from_masses(m1, m2, fstar)
    duration = tau0 + tau1 - tau15 + tau2          # 2PN time from f_* to coalescence
    assert round(duration / 60.0, 1) == dur_min
    assert t0lo <= tau0 <= t0hi and t15lo <= tau15 <= t15hi


@pytest.mark.parametrize("m1,m2,fstar", [(1.4, 1.4, 60.0), (1.0, 3.0, 30.0), (2.2, 1.3, 10.0)])
def test_chirp_time_round_trip(m1, m2, fstar):
    tau0, _, tau15, _ = o.chirp_times_from_masses(m1, m2, fstar)
    x, eta = o.mass_params_from_chirp_times(tau0, tau15, fstar)
    m = x / (math.pi * fstar) / o.T_SUN
    assert m == pytest.approx(m1 + m2, rel=1e-12)
    assert eta == pytest.approx(m1 * m2 / (m1 + m2) ** 2, rel=1e-12)


@pytest.mark.parametrize("m1,m2,fstar", [(1.4, 1.4, 60.0), (1.0, 3.0, 30.0), (3.0, 3.0, 30.0), (1.5, 1.5, 10.0)])
def test_chirp_time_phase_equals_mass_series(m1, m2, fstar):
    """The chirp-time phase equals the textbook TaylorF2 2PN phase written in v = (pi M f)^(1/3)."""
    tau0, _, tau15, _ = o.chirp_times_from_masses(m1, m2, fstar)
    f = np.linspace(fstar * 1.001, 1000.0, 257)
    mass = (m1 + m2) * o.T_SUN
    eta = m1 * m2 / (m1 + m2) ** 2
    v = (math.pi * mass * f) ** (1.0 / 3.0)
    series = (1 + 20.0 / 9.0 * (743.0 / 336.0 + 11.0 / 4.0 * eta) * v ** 2 - 16 * math.pi * v ** 3
              + 10 * (3058673.0 / 1016064.0 + 5429.0 / 1008.0 * eta + 617.0 / 144.0 * eta ** 2) * v ** 4)
    expect = 3.0 / (128.0 * eta) * v ** -5 * series
    got = 2.0 * math.pi * o.chirp_phase_turns(f, tau0, tau15, fstar)
    np.testing.assert_allclose(got, expect, rtol=1e-12, atol=1e-12 * np.abs(expect).max())


def test_template_quadrature_pair_is_orthogonal_and_equal_norm():
    w = sd.SMALL
    setup = _setup(w, sd.make_dataset(w, 0))
    hc = o.template_hc(setup.f, 3.0, 0.3, w.f_low)
    hs = -1j * hc
    for i in range(setup.n_det):
        s = setup.psd_band[i]
        assert abs(o.inner_product(hc, hs, s, setup.df)) < 1e-12 * setup.sigma2[i]
        assert o.inner_product(hs, hs, s, setup.df) == pytest.approx(setup.sigma2[i], rel=1e-13)
        assert o.inner_product(hc, hc, s, setup.df) == pytest.approx(setup.sigma2[i], rel=1e-13)


def test_band_bins_small_grid():
    # N = 16, fs = 16 Hz -> f_k = k Hz; band (2, 6] Hz
    assert list(o.band_bins(16, 16.0, 2.0, 6.0)) == [3, 4, 5, 6]
    assert list(o.band_bins(16, 16.0, 0.0, 100.0)) == [1, 2, 3, 4, 5, 6, 7]    # 0 and N/2 excluded


# ---------------------------------------------------------------- geometry (eq. detresponse)

@pytest.mark.parametrize("alpha,delta,psi", [(0.3, 0.9, 0.0), (2.0, -0.4, 0.7), (4.4, 1.2, 2.5), (5.9, -1.3, 1.1)])
def test_antenna_patterns_polar_detector_closed_form(alpha, delta, psi):
    """Detector at the north pole with arms along ECEF x and y: the textbook
    F+ = 1/2(1+cos^2 th) cos 2ph cos 2ps - cos th sin 2ph sin 2ps,
    Fx = 1/2(1+cos^2 th) cos 2ph sin 2ps + cos th sin 2ph cos 2ps, th = pi/2 - delta, ph = alpha.
    The oracle's basis (-alpha_hat, delta_hat) is the textbook one turned by 90 degrees with psi
    measured the other way, so F_oracle(psi) = -F_textbook(-psi)."""
    det = np.array([[0, 0, 6.4e6, 1, 0, 0, 0, 1, 0]], dtype=float)
    th, ph = math.pi / 2 - delta, alpha

    def textbook(ps):
        a = 0.5 * (1 + math.cos(th) ** 2) * math.cos(2 * ph)
        b = math.cos(th) * math.sin(2 * ph)
        return np.array([a * math.cos(2 * ps) - b * math.sin(2 * ps), a * math.sin(2 * ps) + b * math.cos(2 * ps)])

    got = o.antenna_patterns(det, alpha, delta, psi)[0]
    np.testing.assert_allclose(got, -textbook(-psi), atol=1e-14)
    assert got @ got == pytest.approx(textbook(0.0) @ textbook(0.0), rel=1e-13)


@pytest.mark.parametrize("alpha,delta", [(0.4, 1.5707963267948966), (1.1, 0.9), (3.0, 0.3), (5.2, -0.6), (2.2, 0.0)])
def test_condition_number_of_a_colocated_45_degree_pair(alpha, delta):
    """Two detectors at the north pole, the second with its arms turned by 45 degrees: at polar
    angle th the columns of F are orthogonal with norms (1 + cos^2 th)/2 and |cos th|, so the
    condition number is (1 + cos^2 th) / (2 |cos th|): 1 overhead, +inf in the arms' plane."""
    r = math.sqrt(0.5)
    det = np.array([[0, 0, 6.4e6, 1, 0, 0, 0, 1, 0],
                    [0, 0, 6.4e6, r, r, 0, -r, r, 0]], dtype=float)
    ct = math.cos(math.pi / 2 - delta)
    got = o.condition_number(det, alpha, delta)
    if abs(ct) < 1e-12:
        assert got == math.inf or got > 1e12
    else:
        assert got == pytest.approx((1 + ct * ct) / (2 * abs(ct)), rel=1e-12)


def test_condition_number_single_detector_and_psi_invariance():
    det = sd.detector_geometry()
    assert o.condition_number(det[:1], 1.0, 0.3) == math.inf          # one detector: rank one
    rng = np.random.default_rng(9)
    for _ in range(20):
        a, d, psi = rng.uniform(0, 2 * math.pi), math.asin(rng.uniform(-1, 1)), rng.uniform(0, math.pi)
        s = np.linalg.svd(o.antenna_patterns(det, a, d, psi), compute_uv=False)
        k = o.condition_number(det, a, d)
        assert k >= 1.0 and s[0] / s[1] == pytest.approx(k, rel=1e-12)


def test_delays_bounded_by_baseline_and_tight_along_it():
    det = sd.detector_geometry()
    rng = np.random.default_rng(5)
    for _ in range(50):
        a, d = rng.uniform(0, 2 * math.pi), math.asin(rng.uniform(-1, 1))
        dl = o.arrival_delays(det, a, d)
        for i in range(4):
            for j in range(4):
                assert abs(dl[i] - dl[j]) <= np.linalg.norm(det[i, :3] - det[j, :3]) / o.C_LIGHT * (1 + 1e-12)
    b = det[0, :3] - det[1, :3]                        # source along the H1 - L1 baseline, beyond H1
    b = b / np.linalg.norm(b)
    a, d = math.atan2(b[1], b[0]), math.asin(b[2])
    dl = o.arrival_delays(det, a, d)
    # H1 faces the source: the wave reaches it first, by exactly the baseline light time
    assert dl[1] - dl[0] == pytest.approx(np.linalg.norm(det[0, :3] - det[1, :3]) / o.C_LIGHT, rel=1e-12)


# ---------------------------------------------------------------- t_c scan (Sec. II.C, II.D)

def test_fft_scan_equals_direct_sum_over_every_tc():
    w = dataclasses.replace(sd.SMALL, n_fft=1024, n_samples=900, fs=128.0, f_low=20.0, f_high=60.0)
    setup = _setup(w, sd.make_dataset(w, 3))
    theta = sd.make_particles(w, 3, seed=3)
    for th in theta:
        zf = o.correlations_fft(setup, th)
        zd = o.correlations_direct(setup, th)
        assert np.max(np.abs(zf - zd)) < 1e-10 * np.max(np.abs(zd))
        gf = o.fitness(setup, th)
        gd = o.fitness(setup, th, direct=True)
        assert gf[1] == gd[1] and gf[0] == pytest.approx(gd[0], rel=1e-10)


# ---------------------------------------------------------------- Gamma^2 invariants

@pytest.mark.parametrize("seed", [0, 1, 2, 7])
def test_noiseless_injection_at_truth_gives_snr_squared(seed):
    w = EXACT
    data = sd.make_dataset(w, seed, noise=False)
    setup = _setup(w, data)
    g, t = o.fitness(setup, _truth(w, data["inj"]))
    assert g == pytest.approx(data["inj"]["snr"] ** 2, rel=1e-10)
    assert t == round(data["inj"]["t_c"] * w.fs)


@pytest.mark.parametrize("psi", [0.0, 0.4, 1.3, 2.9])
def test_fitness_invariant_to_injected_polarisation(psi):
    w = EXACT
    data = sd.make_dataset(w, 11, noise=False, psi=psi)
    g, t = o.fitness(_setup(w, data), _truth(w, data["inj"]))
    assert g == pytest.approx(data["inj"]["snr"] ** 2, rel=1e-10)


def test_fitness_invariant_to_antenna_basis():
    """Gamma^2 depends only on the column space of F: U -> F(psi) or U R (R invertible) changes nothing."""
    w = sd.SMALL
    setup = _setup(w, sd.make_dataset(w, 4))
    th = sd.make_particles(w, 1, seed=4)[0]
    z = o.correlations_fft(setup, th)
    u = o.antenna_patterns(setup.det, th[0], th[1], 0.0)
    ref = o.network_statistic(z, u, setup.sigma2)
    for psi in (0.3, 1.9):
        got = o.network_statistic(z, o.antenna_patterns(setup.det, th[0], th[1], psi), setup.sigma2)
        np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12 * ref.max())
    r = np.array([[1.7, -0.4], [0.9, 2.3]])
    np.testing.assert_allclose(o.network_statistic(z, u @ r, setup.sigma2), ref, rtol=1e-10, atol=1e-12 * ref.max())


def test_two_detector_network_is_sum_of_single_detector_snr2():
    """D = 2: F is square and invertible, so Gamma^2 = sum_i (c_i^2 + s_i^2) / sigma_i^2."""
    w = dataclasses.replace(sd.SMALL, detectors=("H1", "V1"))
    setup = _setup(w, sd.make_dataset(w, 5))
    for th in sd.make_particles(w, 3, seed=5):
        z = o.correlations_fft(setup, th)
        got = o.fitness_curve(setup, th)
        expect = np.sum(np.abs(z) ** 2 / setup.sigma2[:, None], axis=0)
        np.testing.assert_allclose(got, expect, rtol=1e-10)


def test_single_detector_is_matched_filter_snr2():
    """D = 1: G is rank one and the rank-1 rule gives the single-detector (c^2 + s^2) / sigma^2."""
    w = dataclasses.replace(sd.SMALL, detectors=("L1",))
    setup = _setup(w, sd.make_dataset(w, 6))
    th = sd.make_particles(w, 1, seed=6)[0]
    z = o.correlations_fft(setup, th)
    np.testing.assert_allclose(o.fitness_curve(setup, th), np.abs(z[0]) ** 2 / setup.sigma2[0], rtol=1e-10)


def test_network_statistic_bounded_by_sum_of_single_detector():
    w = sd.SMALL
    setup = _setup(w, sd.make_dataset(w, 8))
    for th in sd.make_particles(w, 3, seed=8):
        z = o.correlations_fft(setup, th)
        g = o.fitness_curve(setup, th)
        upper = np.sum(np.abs(z) ** 2 / setup.sigma2[:, None], axis=0)
        assert np.all(g >= -1e-12 * upper.max()) and np.all(g <= upper * (1 + 1e-12))


def test_noise_only_statistic_is_chi2_with_four_dof():
    """Gaussian noise, fixed Theta: c_i, s_i ~ N(0, sigma_i^2) independent, so Gamma^2(t) ~ chi^2_4
    (mean 4, variance 8). Pins the noise normalisation, the 4 df factor and sigma_i^2 together."""
    w = dataclasses.replace(sd.C1, n_samples=sd.C1.n_fft)
    means, variances = [], []
    for seed in range(3):
        setup = _setup(w, sd.make_dataset(w, 100 + seed, inject=False))
        th = sd.make_particles(w, 1, seed=seed)[0]
        g = o.fitness_curve(setup, th)
        means.append(g.mean())
        variances.append(g.var())
    assert np.mean(means) == pytest.approx(4.0, abs=0.15)
    assert np.mean(variances) == pytest.approx(8.0, abs=1.2)


# ---------------------------------------------------------------- planted mistakes

def test_pins_catch_a_wrong_delay_sign(monkeypatch):
    w = EXACT
    data = sd.make_dataset(w, 0, noise=False)
    real = o.arrival_delays
    monkeypatch.setattr(o, "arrival_delays", lambda det, a, d: -real(det, a, d))
    g, _ = o.fitness(_setup(w, data), _truth(w, data["inj"]))
    assert g < 0.9 * data["inj"]["snr"] ** 2


def test_pins_catch_a_wrong_tau15_sign(monkeypatch):
    real = o.chirp_coefficients

    def bad(tau0, tau15, f_star):
        c = dict(real(tau0, tau15, f_star))
        c["c15"] = -c["c15"]
        return c

    monkeypatch.setattr(o, "chirp_coefficients", bad)
    with pytest.raises(AssertionError):
        test_chirp_time_phase_equals_mass_series(1.4, 1.4, 60.0)
    w = EXACT
    data = sd.make_dataset(w, 0, noise=False)
    g, _ = o.fitness(_setup(w, data), _truth(w, data["inj"]))
    assert g < 0.9 * data["inj"]["snr"] ** 2


def test_pins_catch_a_wrong_norm_factor(monkeypatch):
    """A template norm off by a factor (e.g. 2 df instead of 4 df) breaks the SNR^2 pin."""
    w = EXACT
    data = sd.make_dataset(w, 2, noise=False)
    setup = _setup(w, data)
    setup.sigma2 = setup.sigma2 * 0.5
    g, _ = o.fitness(setup, _truth(w, data["inj"]))
    assert abs(g / data["inj"]["snr"] ** 2 - 1) > 0.5


def test_pins_catch_a_transposed_antenna_contraction(monkeypatch):
    """Swapping the roles of the detector arms and the wave axes in F breaks the SNR^2 pin."""
    w = EXACT
    data = sd.make_dataset(w, 1, noise=False)
    real = o.antenna_patterns

    def bad(det, a, d, psi=0.0):
        f = real(det, a, d, psi)
        return f[::-1].copy()               # rows attached to the wrong detectors

    monkeypatch.setattr(o, "antenna_patterns", bad)
    g, _ = o.fitness(_setup(w, data), _truth(w, data["inj"]))
    assert g < 0.95 * data["inj"]["snr"] ** 2
