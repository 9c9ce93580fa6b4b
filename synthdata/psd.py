"""Analytic aLIGO noise PSD used for all four detectors of the synthetic network.

S(f) = 1e-49 [x^-4.14 - 5 x^-2 + 111 (1 - x^2 + x^4/2) / (1 + x^2/2)], x = f / 215 Hz
(one-sided, strain^2/Hz). The paper's own curves (Sec. II.A, Fig. 1) are not available, so this
fit stands in for them.
"""

import functools

import numpy as np


def aligo_fit_psd(f):
    f = np.asarray(f, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        x = f / 215.0
        s = 1e-49 * (x ** -4.14 - 5.0 * x ** -2 + 111.0 * (1.0 - x ** 2 + 0.5 * x ** 4) / (1.0 + 0.5 * x ** 2))
    return np.where(f > 0.0, s, np.inf)


@functools.lru_cache(maxsize=8)
def psd_row(n_fft, fs):
    """The fit sampled at f_k = k fs / n_fft for k = 0..n_fft/2 (read-only, cached per grid)."""
    f = np.arange(n_fft // 2 + 1, dtype=np.float64) * (fs / n_fft)
    s = aligo_fit_psd(f)
    s.setflags(write=False)
    return s


@functools.lru_cache(maxsize=8)
def psd_on_grid(n_det, n_fft, fs):
    """PSD sampled at f_k = k fs / n_fft for k = 0..n_fft/2, repeated for every detector: (D, n_fft/2+1)
    (read-only, cached per grid)."""
    s = np.repeat(psd_row(n_fft, fs)[None, :], n_det, axis=0)
    s.setflags(write=False)
    return s
