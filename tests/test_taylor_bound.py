"""The remainder bound behind the FP32 form's shared chirp phase (CPU).

The FP32 pass A forms the chirp phase psi of 4 (or 8) adjacent frequency bins from one anchor bin:
psi(k + c) ~ psi(k) + c psi'(k) + c^2 psi''(k)/2 for c <= C = 3 (or 7), with psi' and psi'' from the
phase's closed form (Sec. II.B: psi/2pi = sum_m c_m phi^-e_m, e_m = 5/3, 1, 2/3, 1/3). The geometry
kernel allows this per particle only when C^3/6 max|psi'''| over the band, bounded term by term at
k_b = f_*/df - 2 (C + 1), is below 1e-7 turns. Checked here against the exact remainder computed from the
oracle's phase in binary64, and against the workloads: the 60-min segments qualify, the short
test segment does not."""

import math

import numpy as np
import pytest

import synthdata as sd
from oracle import fcas_oracle as o

E = (5.0 / 3.0, 1.0, 2.0 / 3.0, 1.0 / 3.0)


def coefficients(tau0, tau15, f_star):
    c = o.chirp_coefficients(tau0, tau15, f_star)
    return (c["c0"], c["c1"], c["c15"], c["c2"])


def bound(cm, f_star, df, cmax=3):
    """The geometry kernel's bound on the remainder of second-order steps of up to cmax bins (turns),
    None if k_b < 1."""
    kb = f_star / df - 2.0 * (cmax + 1)
    if kb < 1.0:
        return None
    r = f_star / (kb * df)
    d3 = sum(abs(c) * e * (e + 1) * (e + 2) * r ** e for c, e in zip(cm, E)) / kb ** 3
    return cmax ** 3 / 6.0 * d3


def exact_remainder(tau0, tau15, f_star, df, k, cmax=3):
    """max over c = 1..cmax of |psi(k + c) - psi(k) - c psi' - c^2 psi''/2| with the derivatives of
    the closed form at bin k (turns)."""
    cm = coefficients(tau0, tau15, f_star)
    bm = [(f_star / (k * df)) ** e for e in E]
    d1 = -sum(e * c * b for e, c, b in zip(E, cm, bm)) / k
    d2 = sum(e * (e + 1) * c * b for e, c, b in zip(E, cm, bm)) / k ** 2
    psi = lambda kk: float(o.chirp_phase_turns(kk * df, tau0, tau15, f_star))
    return max(abs(psi(k + c) - psi(k) - c * d1 - c * c * d2 / 2.0) for c in range(1, cmax + 1))


@pytest.mark.parametrize("cmax", [3, 7])
@pytest.mark.parametrize("w", [sd.C1, sd.SMALL, sd.C2], ids=lambda w: w.name)
def test_bound_dominates_the_exact_remainder(w, cmax):
    df = w.fs / w.n_fft
    f_star = w.f_low
    k_lo = math.ceil(w.f_low / df)
    t0lo, t0hi, t15lo, t15hi = sd.chirp_time_box(f_star)
    for tau0 in np.linspace(t0lo, t0hi, 5):
        for tau15 in np.linspace(t15lo, t15hi, 5):
            b = bound(coefficients(tau0, tau15, f_star), f_star, df, cmax)
            assert b is not None
            for k in (k_lo - cmax, k_lo, k_lo + 17, 2 * k_lo):
                err = exact_remainder(tau0, tau15, f_star, df, k, cmax)
                # binary64 rounding of psi (|psi| < 2e3 turns here) is below 1e-12 turns
                assert err <= b + 1e-12, (w.name, tau0, tau15, k, err, b)


def test_long_segments_qualify_and_the_short_one_does_not():
    for w, box in ((sd.C2, sd.chirp_time_box(sd.C2.f_low)), (sd.PAPER_DNS, sd.PAPER_TAU_BOX)):
        df = w.fs / w.n_fft
        for tau0 in np.linspace(box[0], box[1], 5):
            for tau15 in np.linspace(box[2], box[3], 5):
                assert bound(coefficients(tau0, tau15, w.f_low), w.f_low, df) < 1e-7, (w.name, tau0, tau15)
    w = sd.SMALL
    t0lo, t0hi, t15lo, t15hi = sd.chirp_time_box(w.f_low)
    assert bound(coefficients(t0lo, t15lo, w.f_low), w.f_low, w.fs / w.n_fft) > 1e-7
