"""Plain FP64 CPU oracle of the network GLRT coherent fitness Gamma^2(alpha, delta, tau0, tau1.5).

TEST INFRASTRUCTURE ONLY. This module is imported by the test suite, by the smoke check and by the
benchmark's CPU-baseline / reference arm; the CUDA library never calls it and shares no code with it.

Every step is the paper's definition written out in numpy float64, evaluated naively:

  * data model and detector response  -- Sec. II, eq. detresponse
  * restricted-2PN SPA template        -- Sec. II.B (chirp times tau0, tau1.5; cutoffs f_*, f_high)
  * log-likelihood ratio, inner product -- Sec. II.C, eq. loglikelihood and eq. innprod
  * four-template reparametrisation     -- Sec. II.C (U = F(alpha, delta, 0), h_c, h_s = -i h_c)
  * GLRT fitness, max over A_k and t_c  -- Sec. II.C, eq. gammaSqd
  * precomputed template norms, data-side time shift, over-whitening -- Sec. II.D,
    eq. data_template_innprod

Readings taken where the paper is silent, ambiguous or garbled (each fixed here, with its reason):
  * Gamma^2 = 2 max lambda = X^T M^{-1} X, so that a noiseless injection at the true parameters
    gives the network SNR^2 of eq. optimalSNR (Sec. V compares thresholds of 9.3-9.5 with SNRs of
    9-15, which puts the statistic on the SNR scale).
  * delta is a latitude in [-pi/2, pi/2] (Sec. V's source positions have negative delta);
    n = (cos d cos a, cos d sin a, sin d).
  * Delta^i = -n.r_i / c (eq. detresponse: h^i(t + Delta^i) = F h(t)).
  * The template is zero for f <= f_* (= f_low) and for f > f_high; bins 0 and N/2 are excluded.
  * t_c is the formal TaylorF2 coalescence time at the ECEF origin on the sample grid, the IFFT
    is circular, the maximum is over t in [0, n_samples) with the lowest index on ties.
  * tau1 and tau2 (deferred by the paper to earlier work) are the standard 2PN chirp times.
  * Ill-conditioned G (det G < 1e-12 (tr G / 2)^2): rank-1 projection on G's dominant eigenvector.
"""

import math

import numpy as np

C_LIGHT = 299792458.0
T_SUN = 4.925490947641267e-06  # G Msun / c^3 [s]
RANK1_RTOL = 1e-12


# --------------------------------------------------------------------------------------------
# Frequency grid and band (Sec. II.B cutoffs)
# --------------------------------------------------------------------------------------------

def band_bins(n_fft, fs, f_low, f_high):
    """Bins k with f_low < k fs / N <= f_high and 0 < k < N/2 (template zero for f <= f_*, Sec. II.B)."""
    k = np.arange(n_fft // 2 + 1, dtype=np.int64)
    keep = (k * fs > f_low * n_fft) & (k * fs <= f_high * n_fft) & (k > 0) & (k < n_fft // 2)
    return k[keep]


# --------------------------------------------------------------------------------------------
# Chirp times and the SPA phase (Sec. II.B)
# --------------------------------------------------------------------------------------------

def chirp_times_from_masses(m1, m2, f_star):
    """(tau0, tau1, tau1.5, tau2) [s] of a binary with component masses m1, m2 [Msun] at f_*.
    tau0 and tau1.5 follow Sec. II.B; tau1 and tau2 are the standard 2PN chirp times."""
    m = (m1 + m2) * T_SUN
    eta = m1 * m2 / (m1 + m2) ** 2
    x = math.pi * m * f_star
    tau0 = 5.0 / (256.0 * math.pi * f_star * eta) * x ** (-5.0 / 3.0)
    tau15 = 1.0 / (8.0 * f_star * eta) * x ** (-2.0 / 3.0)
    tau1 = 5.0 / (192.0 * math.pi * f_star * eta * x) * (743.0 / 336.0 + 11.0 * eta / 4.0)
    tau2 = 5.0 / (128.0 * math.pi * f_star * eta * x ** (1.0 / 3.0)) * (
        3058673.0 / 1016064.0 + 5429.0 * eta / 1008.0 + 617.0 * eta ** 2 / 144.0)
    return tau0, tau1, tau15, tau2


def mass_params_from_chirp_times(tau0, tau15, f_star):
    """Invert Sec. II.B's tau0, tau1.5: returns (pi M f_*, eta) with M in seconds.
    tau0 / tau1.5 = 5 / (32 pi) (pi M f_*)^-1 and tau1.5 = (pi M f_*)^(-2/3) / (8 f_* eta)."""
    x = 5.0 * tau15 / (32.0 * math.pi * tau0)
    eta = x ** (-2.0 / 3.0) / (8.0 * f_star * tau15)
    return x, eta


def chirp_coefficients(tau0, tau15, f_star):
    """Coefficients (in turns) of the chirp phase psi(f) / 2pi in powers of phi = f / f_*:
    psi(f) / 2pi = c0 phi^-5/3 + c1 phi^-1 + c15 phi^-2/3 + c2 phi^-1/3, with
    c0 = 3/5 f_* tau0, c1 = f_* tau1, c15 = -3/2 f_* tau1.5, c2 = 3 f_* tau2 (Sec. II.B)."""
    x, eta = mass_params_from_chirp_times(tau0, tau15, f_star)
    tau1 = 5.0 / (192.0 * math.pi * f_star * eta * x) * (743.0 / 336.0 + 11.0 * eta / 4.0)
    tau2 = 5.0 / (128.0 * math.pi * f_star * eta * x ** (1.0 / 3.0)) * (
        3058673.0 / 1016064.0 + 5429.0 * eta / 1008.0 + 617.0 * eta ** 2 / 144.0)
    return dict(c0=0.6 * f_star * tau0, c1=f_star * tau1, c15=-1.5 * f_star * tau15, c2=3.0 * f_star * tau2,
                tau1=tau1, tau2=tau2, eta=eta, x=x)


def chirp_phase_turns(f, tau0, tau15, f_star):
    """psi(f) / 2pi for the template of Sec. II.B (t_c = 0, phi_c = 0 removed)."""
    c = chirp_coefficients(tau0, tau15, f_star)
    phi = np.asarray(f, dtype=np.float64) / f_star
    return (c["c0"] * phi ** (-5.0 / 3.0) + c["c1"] / phi + c["c15"] * phi ** (-2.0 / 3.0)
            + c["c2"] * phi ** (-1.0 / 3.0))


def template_hc(f, tau0, tau15, f_star):
    """h~_c(f) = f^-7/6 exp[-i(psi(f) - pi/4)]: h~_+ of Sec. II.B with A_+ = 1, t_c = 0, phi_c = 0.
    h~_s = h~_x = -i h~_c."""
    f = np.asarray(f, dtype=np.float64)
    psi = 2.0 * math.pi * chirp_phase_turns(f, tau0, tau15, f_star)
    return f ** (-7.0 / 6.0) * np.exp(-1j * (psi - math.pi / 4.0))


# --------------------------------------------------------------------------------------------
# Sky geometry (Sec. II, eq. detresponse)
# --------------------------------------------------------------------------------------------

def sky_vectors(alpha, delta):
    """Unit source direction n and the polarisation basis (X, Y) = (-alpha_hat, delta_hat) at psi = 0."""
    ca, sa, cd, sd = math.cos(alpha), math.sin(alpha), math.cos(delta), math.sin(delta)
    n = np.array([cd * ca, cd * sa, sd])
    x = np.array([sa, -ca, 0.0])
    y = np.array([-sd * ca, -sd * sa, cd])
    return n, x, y


def antenna_patterns(det, alpha, delta, psi=0.0):
    """F(alpha, delta, psi): (D, 2) rows (F+, Fx) = (d : e+, d : ex) with d = (x x^T - y y^T) / 2,
    e+ = X X^T - Y Y^T, ex = X Y^T + Y X^T, the wave axes rotated by psi from (-alpha_hat, delta_hat)."""
    _, bx, by = sky_vectors(alpha, delta)
    wx = math.cos(psi) * bx + math.sin(psi) * by
    wy = -math.sin(psi) * bx + math.cos(psi) * by
    out = np.empty((det.shape[0], 2))
    for i in range(det.shape[0]):
        xa, ya = det[i, 3:6], det[i, 6:9]
        xX, xY, yX, yY = xa @ wx, xa @ wy, ya @ wx, ya @ wy
        out[i, 0] = 0.5 * (xX * xX - xY * xY - yX * yX + yY * yY)
        out[i, 1] = xX * xY - yX * yY
    return out


def condition_number(det, alpha, delta):
    """Condition number of the antenna-pattern matrix F(alpha, delta, psi) (Sec. V: the ill-posedness
    of the network problem at a sky position): the ratio of the largest to the smallest singular
    value of the (D, 2) matrix, by the singular value decomposition. It does not depend on psi,
    which only rotates the columns; +inf when F is (numerically) of rank one, by the rule used for
    G: det(F^T F) < RANK1_RTOL (tr(F^T F) / 2)^2."""
    f = antenna_patterns(det, alpha, delta, 0.0)
    g = f.T @ f
    if g[0, 0] * g[1, 1] - g[0, 1] * g[1, 0] < RANK1_RTOL * (0.5 * (g[0, 0] + g[1, 1])) ** 2:
        return math.inf
    s = np.linalg.svd(f, compute_uv=False)
    return float(s[0] / s[1])


def arrival_delays(det, alpha, delta):
    """Delta^i = -n . r_i / c: the wave reaches detector i Delta^i after the ECEF origin."""
    n, _, _ = sky_vectors(alpha, delta)
    return -(det[:, 0:3] @ n) / C_LIGHT


# --------------------------------------------------------------------------------------------
# Data preparation (Sec. II.D: over-whitening; precomputed template norms)
# --------------------------------------------------------------------------------------------

class OracleSetup:
    """Holds the over-whitened band spectrum and the template norms of one data segment."""

    def __init__(self, det, psd, data, n_fft, fs, f_low, f_high):
        self.det = np.asarray(det, dtype=np.float64)
        self.n_det = self.det.shape[0]
        self.n_fft = int(n_fft)
        self.fs = float(fs)
        self.f_low = float(f_low)
        self.f_high = float(f_high)
        data = np.asarray(data, dtype=np.float64)
        self.n_samples = data.shape[1]
        self.df = self.fs / self.n_fft
        self.k = band_bins(self.n_fft, self.fs, self.f_low, self.f_high)
        self.f = self.k * self.df
        padded = np.zeros((self.n_det, self.n_fft))
        padded[:, : self.n_samples] = data
        xt = np.fft.fft(padded, axis=1)[:, self.k] / self.fs          # x~[k] = dt sum_n x[n] e^{-2 pi i k n/N}
        s = np.asarray(psd, dtype=np.float64)[:, self.k]
        self.psd_band = s
        self.y = xt / s                                                 # over-whitened data
        self.sigma2 = 4.0 * self.df * np.sum(self.f ** (-7.0 / 3.0) / s, axis=1)   # <h_c|h_c>^i = <h_s|h_s>^i


def inner_product(p, q, psd_band, df):
    """<p|q> = 4 Re sum_k p~ q~* / S df on the band (eq. innprod)."""
    return 4.0 * df * np.real(np.sum(p * np.conj(q) / psd_band))


def correlation_spectrum(setup, theta):
    """Q_i[k] = 4 df y~^i[k] e^{2 pi i f_k Delta^i} h~_c*[k] on the band (eq. data_template_innprod)."""
    alpha, delta, tau0, tau15 = (float(v) for v in theta)
    hc = template_hc(setup.f, tau0, tau15, setup.f_low)
    delays = arrival_delays(setup.det, alpha, delta)
    shift = np.exp(2j * math.pi * setup.f[None, :] * delays[:, None])
    return 4.0 * setup.df * setup.y * shift * np.conj(hc)[None, :]


def correlations_fft(setup, theta):
    """Z_i[t] = sum_k Q_i[k] e^{2 pi i k t / N} for t = 0..N-1 by an inverse FFT (the t_c scan).
    c_i = Re Z_i = <x^i(t+Delta^i)|h_c(t - t/fs)>, s_i = -Im Z_i the same for h_s."""
    q = correlation_spectrum(setup, theta)
    full = np.zeros((setup.n_det, setup.n_fft), dtype=np.complex128)
    full[:, setup.k] = q
    return np.fft.ifft(full, axis=1) * setup.n_fft


def correlations_direct(setup, theta):
    """Same Z_i[t] by a brute-force sum over every bin for every t (small N only)."""
    q = correlation_spectrum(setup, theta)
    n = setup.n_fft
    t = np.arange(n)
    out = np.zeros((setup.n_det, n), dtype=np.complex128)
    for j, kk in enumerate(setup.k):
        out += q[:, j : j + 1] * np.exp(2j * math.pi * ((kk * t) % n) / n)[None, :]
    return out


# --------------------------------------------------------------------------------------------
# Maximisation over the amplitudes A_k (Sec. II.C) and over t_c
# --------------------------------------------------------------------------------------------

def projection_matrix(u, sigma2):
    """G^-1 for G = sum_i sigma_i^2 U^i U^i^T (the 2x2 block of the 4x4 template Gram matrix, which is
    diag(G, G) because <h_c|h_s> = 0 and <h_s|h_s> = <h_c|h_c>). If G is numerically singular the
    rank-1 pseudo-inverse e e^T / lambda_max is returned instead."""
    g = (u * sigma2[:, None]).T @ u
    det = g[0, 0] * g[1, 1] - g[0, 1] * g[1, 0]
    tr = g[0, 0] + g[1, 1]
    if det < RANK1_RTOL * (0.5 * tr) ** 2:
        w, v = np.linalg.eigh(g)
        e = v[:, 1]
        return np.outer(e, e) / w[1]
    return np.array([[g[1, 1], -g[0, 1]], [-g[1, 0], g[0, 0]]]) / det


def network_statistic(z, u, sigma2):
    """Gamma^2(t) = X_c^T G^-1 X_c + X_s^T G^-1 X_s, X_c = sum_i U^i c_i, X_s = sum_i U^i s_i
    (= 2 max over A_k of the log-likelihood ratio at fixed t_c)."""
    ginv = projection_matrix(u, sigma2)
    c = np.real(z)
    s = -np.imag(z)
    xc = u.T @ c
    xs = u.T @ s
    return np.einsum("at,ab,bt->t", xc, ginv, xc) + np.einsum("at,ab,bt->t", xs, ginv, xs)


def fitness_curve(setup, theta, direct=False):
    alpha, delta = float(theta[0]), float(theta[1])
    z = correlations_direct(setup, theta) if direct else correlations_fft(setup, theta)
    u = antenna_patterns(setup.det, alpha, delta, 0.0)
    return network_statistic(z, u, setup.sigma2)


def fitness(setup, theta, direct=False):
    """(Gamma^2 = max over t in [0, n_samples) of Gamma^2(t), argmax t with the lowest index on ties)."""
    g = fitness_curve(setup, theta, direct=direct)[: setup.n_samples]
    t = int(np.argmax(g))
    return float(g[t]), t


def fitness_batch(setup, thetas):
    out_f = np.empty(len(thetas))
    out_t = np.empty(len(thetas), dtype=np.int64)
    for j, th in enumerate(thetas):
        out_f[j], out_t[j] = fitness(setup, th)
    return out_f, out_t


# --------------------------------------------------------------------------------------------
# Gradient of Gamma^2 at a fixed t_c (envelope theorem: the argmax over t_c is held fixed)
# --------------------------------------------------------------------------------------------

def _statistic_at(setup, theta, t):
    """Gamma^2(theta, t) at one t_c with only real-analytic operations (direct sums with cos and
    sin, no FFT, no conjugation), so that it accepts complex theta for complex-step derivatives."""
    alpha, delta, tau0, tau15 = theta
    ca, sa, cd, sd = np.cos(alpha), np.sin(alpha), np.cos(delta), np.sin(delta)
    n = np.array([cd * ca, cd * sa, sd])
    bx = np.array([sa, -ca, 0.0 * sa])
    by = np.array([-sd * ca, -sd * sa, cd])
    f_star = setup.f_low
    x = 5.0 * tau15 / (32.0 * math.pi * tau0)
    eta = x ** (-2.0 / 3.0) / (8.0 * f_star * tau15)
    tau1 = 5.0 / (192.0 * math.pi * f_star * eta * x) * (743.0 / 336.0 + 11.0 * eta / 4.0)
    tau2 = 5.0 / (128.0 * math.pi * f_star * eta * x ** (1.0 / 3.0)) * (
        3058673.0 / 1016064.0 + 5429.0 * eta / 1008.0 + 617.0 * eta ** 2 / 144.0)
    phi = setup.f / f_star
    psi_turns = (0.6 * f_star * tau0 * phi ** (-5.0 / 3.0) + f_star * tau1 / phi
                 - 1.5 * f_star * tau15 * phi ** (-2.0 / 3.0) + 3.0 * f_star * tau2 * phi ** (-1.0 / 3.0))
    amp = 4.0 * setup.df * setup.f ** (-7.0 / 6.0)
    shift = (setup.k * t % setup.n_fft) / setup.n_fft          # e^{2 pi i k t / N}, exact turns
    u = []
    cs = []
    ss = []
    for i in range(setup.n_det):
        xa, ya = setup.det[i, 3:6], setup.det[i, 6:9]
        xX, xY, yX, yY = xa @ bx, xa @ by, ya @ bx, ya @ by
        u.append((0.5 * (xX * xX - xY * xY - yX * yX + yY * yY), xX * xY - yX * yY))
        delay = -(setup.det[i, 0:3] @ n) / C_LIGHT
        # Q = 4 df y~ e^{2 pi i f Delta} h~_c*, h~_c* = f^-7/6 e^{i(psi - pi/4)}; times e^{2 pi i k t / N}
        ph = 2.0 * math.pi * (psi_turns + setup.f * delay + shift) - math.pi / 4.0
        yr, yi = np.real(setup.y[i]), np.imag(setup.y[i])
        re = amp * (yr * np.cos(ph) - yi * np.sin(ph))
        im = amp * (yr * np.sin(ph) + yi * np.cos(ph))
        cs.append(np.sum(re))          # c_i = Re Z_i
        ss.append(-np.sum(im))         # s_i = -Im Z_i
    g11 = sum(setup.sigma2[i] * u[i][0] * u[i][0] for i in range(setup.n_det))
    g12 = sum(setup.sigma2[i] * u[i][0] * u[i][1] for i in range(setup.n_det))
    g22 = sum(setup.sigma2[i] * u[i][1] * u[i][1] for i in range(setup.n_det))
    det = g11 * g22 - g12 * g12
    xc = (sum(u[i][0] * cs[i] for i in range(setup.n_det)), sum(u[i][1] * cs[i] for i in range(setup.n_det)))
    xs = (sum(u[i][0] * ss[i] for i in range(setup.n_det)), sum(u[i][1] * ss[i] for i in range(setup.n_det)))
    quad = lambda v: (g22 * v[0] * v[0] - 2.0 * g12 * v[0] * v[1] + g11 * v[1] * v[1]) / det
    return quad(xc) + quad(xs)


def statistic_at(setup, theta, t):
    """Gamma^2(theta, t) at a single t_c (real)."""
    return float(np.real(_statistic_at(setup, [complex(v) for v in theta], int(t))))


def gradient(setup, theta, t, h=1e-30):
    """d Gamma^2(theta, t) / d theta at fixed t by the complex-step derivative
    Im f(theta + i h e_j) / h (exact to rounding for a real-analytic f; full-rank G only)."""
    g = np.empty(4)
    for j in range(4):
        th = [complex(v) for v in theta]
        th[j] += 1j * h
        g[j] = np.imag(_statistic_at(setup, th, int(t))) / h
    return g
