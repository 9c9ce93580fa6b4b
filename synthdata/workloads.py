"""Workload descriptions and seeded data generation.

Noise: stationary Gaussian with one-sided PSD S (Sec. II.A), drawn in the frequency domain at the
FFT length N with E|n~_k|^2 = T S(f_k)/2 (T = N/fs) on the analysis band, zero elsewhere, then
transformed to a real time series; the first ``n_samples`` samples are kept (for the 60-min case
the rest of the 2^23 grid is the zero padding).

Injection: the H1 data model of Sec. II (x = h + n) with the detector response of eq. detresponse,
h^i(t) = F+^i h+(t - D^i) + Fx^i hx(t - D^i), D^i = -n.r_i / c, and the restricted-2PN stationary
phase polarisations of Sec. II.B. The phase is written here in its mass form (the TaylorF2
v-series in M and eta), independently of the chirp-time form the fitness code uses; the
amplitude is set so that the network SNR of eq. optimalSNR takes the requested value.

Particles: alpha ~ U[0, 2pi), sin(delta) ~ U[-1, 1], (tau0, tau1.5) uniform over the rectangle
spanned by component masses 1..3 Msun at the lower cutoff.

All draws use numpy's counter-based Philox generator, so a seed gives the same inputs on any host.
"""

import dataclasses
import math

import numpy as np

from .psd import aligo_fit_psd, psd_on_grid, psd_row
from .sites import detector_geometry

C_LIGHT = 299792458.0
T_SUN = 4.925490947641267e-06  # G Msun / c^3 [s]


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    fs: float
    n_samples: int
    n_fft: int
    f_low: float
    f_high: float
    m1: float
    m2: float
    snr: float
    arrival_s: float
    n_particles: int
    detectors: tuple = ("H1", "L1", "V1", "K1")

    @property
    def n_det(self):
        return len(self.detectors)


# Small case the oracle finishes in well under a second (used by many parity tests).
SMALL = Workload("small-4det-4096", fs=512.0, n_samples=3000, n_fft=4096, f_low=80.0, f_high=250.0,
                 m1=1.4, m2=1.4, snr=12.0, arrival_s=0.5, n_particles=24)
# 4 det x 64 s @ 1024 Hz, band 60-500 Hz, 40 particles.
C1 = Workload("4det-64s-1024Hz", fs=1024.0, n_samples=65536, n_fft=65536, f_low=60.0, f_high=500.0,
              m1=1.4, m2=1.4, snr=12.0, arrival_s=64.0 / 3.0, n_particles=40)
# 4 det x 60 min @ 2048 Hz (7,372,800 samples zero-padded to 2^23), band 30-1000 Hz, 320 particles.
C2 = Workload("4det-60min-2048Hz", fs=2048.0, n_samples=7372800, n_fft=1 << 23, f_low=30.0, f_high=1000.0,
              m1=1.4, m2=1.4, snr=10.0, arrival_s=1200.0, n_particles=320)

# The paper's own search configuration (Sec. V): 4 det x 60 min @ 2048 Hz with f_* = 10 Hz, an
# equal-mass 1.5 + 1.5 Msun signal arriving 20 min into the data (it lasts 15.1 min from 10 Hz),
# searched over tau0 in [500, 1500] s, tau1.5 in [5, 15] s; SNR 12.
PAPER_DNS = Workload("4det-60min-2048Hz-fstar10", fs=2048.0, n_samples=7372800, n_fft=1 << 23, f_low=10.0,
                     f_high=1000.0, m1=1.5, m2=1.5, snr=12.0, arrival_s=1200.0, n_particles=40)
PAPER_TAU_BOX = (500.0, 1500.0, 5.0, 15.0)

_BY_NAME = {w.name: w for w in (SMALL, C1, C2, PAPER_DNS)}


def workload_by_name(name):
    return _BY_NAME[name]


def _rng(seed, stream):
    return np.random.Generator(np.random.Philox(key=[int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream)]))


def _band_mask(n_fft, fs, f_low, f_high):
    k = np.arange(n_fft // 2 + 1)
    # f_low < k fs / N <= f_high, 0 < k < N/2, compared in exact products
    return (k * fs > f_low * n_fft) & (k * fs <= f_high * n_fft) & (k > 0) & (k < n_fft // 2)


def _chirp_times_tau0_tau15(m1, m2, f_star):
    m = (m1 + m2) * T_SUN
    eta = m1 * m2 / (m1 + m2) ** 2
    x = math.pi * m * f_star
    tau0 = 5.0 / (256.0 * math.pi * f_star * eta) * x ** (-5.0 / 3.0)
    tau15 = 1.0 / (8.0 * f_star * eta) * x ** (-2.0 / 3.0)
    return tau0, tau15


def chirp_time_box(f_star, m_lo=1.0, m_hi=3.0):
    """(tau0_min, tau0_max, tau15_min, tau15_max): both chirp times fall monotonically with the
    masses on the square [m_lo, m_hi]^2, so the corners (m_hi, m_hi) and (m_lo, m_lo) bound them."""
    t0a, t15a = _chirp_times_tau0_tau15(m_hi, m_hi, f_star)
    t0b, t15b = _chirp_times_tau0_tau15(m_lo, m_lo, f_star)
    return (t0a, t0b, t15a, t15b)


def _taylorf2_phase(f, m1, m2):
    """Restricted-2PN SPA phase psi(f) in its (M, eta) v-series form [rad]."""
    m = (m1 + m2) * T_SUN
    eta = m1 * m2 / (m1 + m2) ** 2
    v = (math.pi * m * f) ** (1.0 / 3.0)
    series = (1.0
              + (20.0 / 9.0) * (743.0 / 336.0 + 11.0 * eta / 4.0) * v ** 2
              - 16.0 * math.pi * v ** 3
              + 10.0 * (3058673.0 / 1016064.0 + 5429.0 * eta / 1008.0 + 617.0 * eta ** 2 / 144.0) * v ** 4)
    return 3.0 / (128.0 * eta * v ** 5) * series


def _time_to_coalescence(m1, m2, f):
    """SPA time-to-coalescence at frequency f: -(1/2pi) dpsi/df (central difference)."""
    h = f * 1e-6
    return -(_taylorf2_phase(f + h, m1, m2) - _taylorf2_phase(f - h, m1, m2)) / (2.0 * h) / (2.0 * math.pi)


def _response(det_row, alpha, delta, psi):
    """(F+, Fx, delay) of one detector for a source at (alpha, delta) with polarisation angle psi,
    written as a full tensor contraction in the wave frame."""
    r, xa, ya = det_row[0:3], det_row[3:6], det_row[6:9]
    n_hat = np.array([math.cos(delta) * math.cos(alpha), math.cos(delta) * math.sin(alpha), math.sin(delta)])
    m_hat = np.array([math.sin(alpha), -math.cos(alpha), 0.0])  # -alpha_hat
    l_hat = np.array([-math.sin(delta) * math.cos(alpha), -math.sin(delta) * math.sin(alpha), math.cos(delta)])
    p_hat = math.cos(psi) * m_hat + math.sin(psi) * l_hat
    q_hat = -math.sin(psi) * m_hat + math.cos(psi) * l_hat
    e_plus = np.outer(p_hat, p_hat) - np.outer(q_hat, q_hat)
    e_cross = np.outer(p_hat, q_hat) + np.outer(q_hat, p_hat)
    d = 0.5 * (np.outer(xa, xa) - np.outer(ya, ya))
    return float(np.einsum("ab,ab->", d, e_plus)), float(np.einsum("ab,ab->", d, e_cross)), -float(n_hat @ r) / C_LIGHT


def injection_spectrum(w, det, psd, params):
    """Frequency-domain detector responses h~^i[k] (D, N/2+1) on the analysis band, normalised to
    the requested network SNR with the discrete inner product 4 df sum |h~|^2 / S."""
    n = w.n_fft
    mask = _band_mask(n, w.fs, w.f_low, w.f_high)
    k = np.nonzero(mask)[0]
    f = k * (w.fs / n)
    big_psi = (2.0 * math.pi * f * params["t_c"] - params["phi_c"] - math.pi / 4.0
               + _taylorf2_phase(f, params["m1"], params["m2"]))
    amp = f ** (-7.0 / 6.0)
    cos_i = params["cos_iota"]
    h_plus = 0.5 * (1.0 + cos_i ** 2) * amp * np.exp(-1j * big_psi)
    h_cross = cos_i * amp * np.exp(-1j * (big_psi + math.pi / 2.0))
    out = np.zeros((det.shape[0], n // 2 + 1), dtype=np.complex128)
    for i in range(det.shape[0]):
        fp, fx, delay = _response(det[i], params["alpha"], params["delta"], params["psi"])
        out[i, k] = (fp * h_plus + fx * h_cross) * np.exp(-2j * math.pi * f * delay)
    df = w.fs / n
    snr2 = sum(4.0 * df * np.sum(np.abs(out[i, k]) ** 2 / psd[i, k]) for i in range(det.shape[0]))
    return out * (params["snr"] / math.sqrt(snr2))


def injection_params(w, seed, snr=None, on_grid=True):
    g = _rng(seed, 1)
    alpha = g.uniform(0.0, 2.0 * math.pi)
    delta = math.asin(g.uniform(-1.0, 1.0))
    psi = g.uniform(0.0, math.pi)
    cos_iota = g.uniform(-1.0, 1.0)
    phi_c = g.uniform(0.0, 2.0 * math.pi)
    t_c = w.arrival_s + _time_to_coalescence(w.m1, w.m2, w.f_low)
    if on_grid:
        t_c = round(t_c * w.fs) / w.fs
    return dict(alpha=alpha, delta=delta, psi=psi, cos_iota=cos_iota, phi_c=phi_c, t_c=t_c,
                m1=w.m1, m2=w.m2, snr=w.snr if snr is None else snr)


def noise_spectrum(w, seed, n_det):
    """Coloured Gaussian noise n~^i[k] (D, N/2+1) with E|n~|^2 = T S / 2 on the analysis band."""
    n = w.n_fft
    mask = _band_mask(n, w.fs, w.f_low, w.f_high)
    k = np.nonzero(mask)[0]
    t_pad = n / w.fs
    s = psd_row(n, w.fs)[k]
    out = np.zeros((n_det, n // 2 + 1), dtype=np.complex128)
    for i in range(n_det):
        g = _rng(seed, 100 + i)
        sd = np.sqrt(t_pad * s / 4.0)
        out[i, k] = sd * (g.standard_normal(k.size) + 1j * g.standard_normal(k.size))
    return out


def spectrum_to_series(w, spec):
    """Real time series x[n] whose DFT dt * sum_n x[n] e^{-2 pi i k n / N} equals ``spec`` on
    0 <= k <= N/2 (Hermitian completion), truncated to the first ``n_samples`` samples."""
    dt = 1.0 / w.fs
    x = np.fft.irfft(spec, n=w.n_fft, axis=-1) / dt
    return np.ascontiguousarray(x[:, : w.n_samples])


def make_dataset(w, seed=0, noise=True, inject=True, snr=None, psi=None):
    """Return dict with data (D, n_samples), psd (D, N/2+1), det (D, 9) and the injection params."""
    det = detector_geometry(w.detectors)
    psd = psd_on_grid(w.n_det, w.n_fft, w.fs)
    spec = np.zeros((w.n_det, w.n_fft // 2 + 1), dtype=np.complex128)
    params = injection_params(w, seed, snr=snr)
    if psi is not None:
        params["psi"] = psi
    if noise:
        spec += noise_spectrum(w, seed, w.n_det)
    if inject:
        spec += injection_spectrum(w, det, psd, params)
    data = spectrum_to_series(w, spec)
    return dict(data=data, psd=psd, det=det, inj=params if inject else None)


def make_particles(w, n=None, seed=0, f_star=None):
    """(n, 4) array of (alpha, delta, tau0, tau1.5) drawn uniformly over the sky and the chirp-time box."""
    n = w.n_particles if n is None else n
    f_star = w.f_low if f_star is None else f_star
    g = _rng(seed, 2)
    t0lo, t0hi, t15lo, t15hi = chirp_time_box(f_star)
    alpha = g.uniform(0.0, 2.0 * math.pi, n)
    delta = np.arcsin(g.uniform(-1.0, 1.0, n))
    tau0 = g.uniform(t0lo, t0hi, n)
    tau15 = g.uniform(t15lo, t15hi, n)
    return np.ascontiguousarray(np.stack([alpha, delta, tau0, tau15], axis=1))
