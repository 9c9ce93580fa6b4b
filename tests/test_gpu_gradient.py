"""GPU adjoint gradient of the coherent fitness at fixed t_c against the oracle's FP64 gradient
(complex step) and central finite differences; the torch.autograd path; gradient polishing."""

import numpy as np
import pytest

import synthdata as sd
from oracle import fcas_oracle as o
from parity_util import make_ctx, oracle_setup

pytestmark = pytest.mark.gpu

# Per-component tolerance of the adjoint gradient. The adjoint reduces, per detector and band bin, the
# term Q_i[k] e^{2 pi i k t/N} (and its products with k and the chirp-basis powers, which are exact
# binary64 weights) in binary64; its error is that of each term, a relative error of at most
# EPS_TERM[form] made independently in every bin:
#   FP32: the phase is the FP32 sum of five float-float fractions (each within a few 2^-24 turn) and
#         the bin's shift, sin/cos in FP32, the product Y e^{i phase} in FP32: |error| <= ~1e-6;
#   binary64 and float-float: the phase reaches c_0 phi^-5/3 ~ 2e3 turns on these workloads and is
#         formed in binary64 before its reduction: 2 pi 2e3 2^-53 ~ 1.4e-12 (1e-11 with margin).
# A gradient component is a fixed binary64 combination of such sums, so its error is bounded by
# perturbing every term of the oracle by a random relative error of that size and taking the largest
# change of the oracle's own (complex-step) gradient over a few draws, times SAFETY for the random
# draw's shortfall against the worst case, plus REL_FLOOR of the component for the binary64 rounding
# of the combination itself.
EPS_TERM = {"fp32": 1e-6, "fp64": 1e-11, "ff": 1e-11}
SAFETY = 8.0
REL_FLOOR = {"fp32": 1e-6, "fp64": 1e-10, "ff": 1e-10}
DRAWS = 3


_SPREAD = {}


def component_tolerance(setup, theta, t, precision, seed=0):
    """(oracle gradient, per-component tolerance) at (theta, t) for the given form. The gradient's
    response to the per-term errors is linear in their size (first order), so the spread is taken once
    per point for errors of size EPS0 and scaled to each form's EPS_TERM."""
    eps0 = 1e-6
    key = (id(setup), tuple(float(v) for v in theta), int(t), seed)
    if key not in _SPREAD:
        rng = np.random.default_rng(seed)
        g0 = o.gradient(setup, theta, t)
        y0 = setup.y
        spread = np.zeros(4)
        try:
            for _ in range(DRAWS):
                d = (rng.standard_normal(y0.shape) + 1j * rng.standard_normal(y0.shape)) * (eps0 / np.sqrt(2))
                setup.y = y0 * (1.0 + d)
                spread = np.maximum(spread, np.abs(o.gradient(setup, theta, t) - g0))
        finally:
            setup.y = y0
        _SPREAD[key] = (g0, spread)
    g0, spread = _SPREAD[key]
    return g0, SAFETY * spread * (EPS_TERM[precision] / eps0) + REL_FLOOR[precision] * np.abs(g0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_02150_gb300 import build as b
    b.build()


def _gpu_grad(ctx, theta):
    import paper_2002_02150_gb300 as fc
    f, tc = fc.fcas_fitness(ctx, theta)
    g = fc.fcas_gradient(ctx, theta, tc)
    return np.asarray(f), np.asarray(tc), np.asarray(g)


def _check(setup, theta, tc, g, precision, context):
    for j in range(len(theta)):
        ref, tol = component_tolerance(setup, theta[j], tc[j], precision, seed=j)
        err = np.abs(g[j] - ref)
        assert np.all(err <= tol), f"{context} particle {j}: {g[j]} vs {ref} (|error| {err}, tolerance {tol})"


@pytest.mark.parametrize("precision", ["fp32", "fp64", "ff"])
def test_gradient_matches_oracle_small(precision):
    w = sd.SMALL
    data = sd.make_dataset(w, 7)
    theta = sd.make_particles(w, 12, seed=7)
    with make_ctx(w, data, precision) as ctx:
        f, tc, g = _gpu_grad(ctx, theta)
    _check(oracle_setup(w, data), theta, tc, g, precision, "SMALL")


def test_gradient_320_particles_64s_fp32():
    """The differentiation workload: 320 particles on the 64-s data, FP32 form."""
    w = sd.C1
    data = sd.make_dataset(w, 0)
    theta = sd.make_particles(w, 320, seed=1)
    with make_ctx(w, data, "fp32") as ctx:
        f, tc, g = _gpu_grad(ctx, theta)
    setup = oracle_setup(w, data)
    assert np.all(np.isfinite(g))
    _check(setup, theta[::8], tc[::8], g[::8], "fp32", "64s")


@pytest.mark.parametrize("rel_step", [1e-6, 1e-5, 1e-4, 1e-3])
def test_gradient_against_fp64_central_differences(rel_step):
    w = sd.C1
    data = sd.make_dataset(w, 0)
    theta = sd.make_particles(w, 2, seed=3)
    setup = oracle_setup(w, data)
    with make_ctx(w, data, "fp32") as ctx:
        f, tc, g = _gpu_grad(ctx, theta)
    tols = [component_tolerance(setup, theta[j], tc[j], "fp32", seed=j)[1] for j in range(2)]
    for j in range(2):
        scale = np.array([1.0, 1.0, theta[j, 2], theta[j, 3]])
        for m in range(4):
            h = rel_step * scale[m]
            e = np.zeros(4)
            e[m] = h
            fd = lambda hh: (o.statistic_at(setup, theta[j] + e * hh / h, tc[j])
                             - o.statistic_at(setup, theta[j] - e * hh / h, tc[j])) / (2 * hh)
            d_h, d_h2 = fd(h), fd(h / 2)
            # truncation error of the central difference, from its own Richardson estimate, plus the
            # FP32 adjoint's own per-component tolerance and the rounding of the differenced values
            trunc = 2.0 * abs(d_h - d_h2)
            tol = tols[j][m] + trunc + 1e-13 * abs(f[j]) / h
            assert abs(d_h - g[j, m]) <= tol, (j, m, d_h, g[j, m], tol)


def test_autograd_function_uses_the_adjoint():
    import torch
    import paper_2002_02150_gb300 as fc
    w = sd.SMALL
    data = sd.make_dataset(w, 8)
    theta = torch.tensor(sd.make_particles(w, 5, seed=8), device="cuda:0", requires_grad=True)
    with make_ctx(w, data, "fp32") as ctx:
        fit, tc = fc.coherent_fitness(ctx, theta)
        (2.0 * fit).sum().backward()
        g = fc.fcas_gradient(ctx, theta.detach(), tc)
    torch.testing.assert_close(theta.grad, 2.0 * g)


def test_polish_improves_pso_best_particles_judged_by_the_oracle():
    """10 gradient-polish steps (fcas_polish, one call per step) on each PSO run's best particle, every
    step judged by the FP64 oracle: the oracle's fitness never falls by more than the FP32 form's
    parity tolerance from one step to the next, and it rises over the 10 steps on some runs."""
    import paper_2002_02150_gb300 as fc
    from parity_util import RTOL
    w = sd.C1
    data = sd.make_dataset(w, 0)
    setup = oracle_setup(w, data)
    t0lo, t0hi, t15lo, t15hi = sd.chirp_time_box(w.f_low)
    cfg = fc.pso_config(n_runs=4, n_particles=40, n_iter=80, seed=4,
                        box=(0.0, 2 * np.pi, -0.5 * np.pi, 0.5 * np.pi, t0lo, t0hi, t15lo, t15hi))
    with make_ctx(w, data, "fp32") as ctx:
        res = fc.fcas_search(ctx, cfg)
        theta = np.array([r["theta"] for r in res])
        oracle = lambda th: np.array([o.fitness(setup, t)[0] for t in th])
        first = prev = oracle(theta)
        total = np.zeros(len(theta), dtype=np.int64)
        for _ in range(10):
            theta, fit, tc, acc = fc.fcas_polish(ctx, theta, steps=1)
            now = oracle(theta)
            assert np.all(now >= prev * (1.0 - RTOL["fp32"])), (prev, now)
            np.testing.assert_allclose(fit, now, rtol=RTOL["fp32"])
            total += acc
            prev = now
    assert np.any(prev > first) and np.any(total > 0)


def test_polish_in_one_call_equals_step_by_step():
    """fcas_polish with steps = 3 gives the points, fitness and t_c of three one-step calls, on host
    and on device arrays."""
    import torch
    import paper_2002_02150_gb300 as fc
    w = sd.SMALL
    data = sd.make_dataset(w, 9)
    theta = sd.make_particles(w, 6, seed=9)
    with make_ctx(w, data, "fp32") as ctx:
        f0, _ = fc.fcas_fitness(ctx, theta)
        th3, f3, t3, a3 = fc.fcas_polish(ctx, theta, steps=3)
        th, acc = theta.copy(), np.zeros(6, dtype=np.int32)
        for _ in range(3):
            th, f1, t1, a1 = fc.fcas_polish(ctx, th, steps=1)
            acc += a1
        thd, fd, tcd, ad = fc.fcas_polish(ctx, torch.tensor(theta, device="cuda:0"), steps=3)
    np.testing.assert_array_equal(th3, th)
    np.testing.assert_array_equal(f3, f1)
    np.testing.assert_array_equal(t3, t1)
    np.testing.assert_array_equal(a3, acc)
    np.testing.assert_array_equal(thd.cpu().numpy(), th3)
    np.testing.assert_array_equal(ad.cpu().numpy(), a3)
    assert np.all(f3 >= f0)


def test_gradient_60min_sampled():
    """The 60-min workload (N = 2^23): the adjoint gradient of two particles in both forms against
    the oracle's complex-step gradient at the same t_c."""
    w = sd.C2
    data = sd.make_dataset(w, 0)
    theta = sd.make_particles(w, 2, seed=5)
    setup = oracle_setup(w, data)
    for precision in ("fp32", "fp64"):
        with make_ctx(w, data, precision) as ctx:
            f, tc, g = _gpu_grad(ctx, theta)
        _check(setup, theta, tc, g, precision, f"60min {precision}")
