"""GPU adjoint gradient of the coherent fitness at fixed t_c against the oracle's FP64 gradient
(complex step) and central finite differences; the torch.autograd path; gradient polishing."""

import numpy as np
import pytest

import synthdata as sd
from oracle import fcas_oracle as o
from parity_util import make_ctx, oracle_setup

pytestmark = pytest.mark.gpu

GRAD_RTOL = {"fp32": 2e-3, "fp64": 1e-8, "ff": 1e-8}


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
        ref = o.gradient(setup, theta[j], tc[j])
        scale = np.abs(ref).max()
        err = np.abs(g[j] - ref).max()
        assert err <= GRAD_RTOL[precision] * scale, f"{context} particle {j}: {g[j]} vs {ref}"


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
    for j in range(2):
        scale = np.array([1.0, 1.0, theta[j, 2], theta[j, 3]])
        for m in range(4):
            h = rel_step * scale[m]
            e = np.zeros(4)
            e[m] = h
            fd = lambda hh: (o.statistic_at(setup, theta[j] + e * hh / h, tc[j])
                             - o.statistic_at(setup, theta[j] - e * hh / h, tc[j])) / (2 * hh)
            d_h, d_h2 = fd(h), fd(h / 2)
            # truncation error of the central difference, from its own Richardson estimate
            trunc = 2.0 * abs(d_h - d_h2)
            tol = (GRAD_RTOL["fp32"] + 1e-7) * np.abs(g[j]).max() + trunc
            assert abs(d_h - g[j, m]) <= tol, (j, m, d_h, g[j, m])


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


def test_polish_improves_pso_best_particles_measured_by_the_oracle():
    """10 gradient-polish steps on each run's best particle; steps are accepted only when the FP64
    oracle's fitness increases, so the gain the oracle measures is >= 0 and positive on some runs."""
    import paper_2002_02150_gb300 as fc
    w = sd.C1
    data = sd.make_dataset(w, 0)
    setup = oracle_setup(w, data)
    t0lo, t0hi, t15lo, t15hi = sd.chirp_time_box(w.f_low)
    cfg = fc.pso_config(n_runs=4, n_particles=40, n_iter=80, seed=4,
                        box=(0.0, 2 * np.pi, -0.5 * np.pi, 0.5 * np.pi, t0lo, t0hi, t15lo, t15hi))
    with make_ctx(w, data, "fp32") as ctx:
        res = fc.fcas_search(ctx, cfg)
        theta = np.array([r["theta"] for r in res])
        before = np.array([o.fitness(setup, th)[0] for th in theta])
        by_oracle = lambda th: tuple(np.array(v) for v in zip(*[o.fitness(setup, t) for t in th]))
        th2, after, acc = fc.polish(ctx, theta, steps=10, evaluate=by_oracle)
    assert np.all(after >= before)
    assert np.any(after > before)


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
