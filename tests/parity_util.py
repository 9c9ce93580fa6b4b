"""Helpers shared by the GPU parity tests: build the oracle and the library context on the same
seeded inputs and compare fitness and argmax element by element."""

import numpy as np

from oracle import fcas_oracle as o

# Parity tolerance of the FP32 form (float-float phase): |Gamma^2_GPU - Gamma^2_oracle| / Gamma^2_oracle
# <= 1e-4, argmax equal or a tie within 1e-5; the binary64 and float-float forms are held much tighter.
RTOL = {"fp32": 1e-4, "fp64": 1e-9, "ff": 1e-9}
TIE_RTOL = 1e-5


def oracle_setup(w, data):
    return o.OracleSetup(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high)


def make_ctx(w, data, precision, max_batch=0):
    import paper_2002_02150_gb300 as fc
    return fc.fcas_create(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high,
                          precision=precision, max_batch=max_batch)


def gpu_fitness(ctx, theta):
    import torch
    import paper_2002_02150_gb300 as fc
    th = torch.tensor(np.asarray(theta, dtype=np.float64), device="cuda:0")
    fit, tc = fc.fcas_fitness(ctx, th)
    torch.cuda.synchronize()
    return fit.cpu().numpy(), tc.cpu().numpy()


def assert_parity(setup, theta, fit, tc, precision, context=""):
    """Same Gamma^2 within the form's tolerance and the same argmax, or a tie within TIE_RTOL."""
    for j, th in enumerate(theta):
        curve = o.fitness_curve(setup, th)[: setup.n_samples]
        t_ref = int(np.argmax(curve))
        g_ref = float(curve[t_ref])
        rel = abs(fit[j] - g_ref) / g_ref
        assert rel <= RTOL[precision], f"{context} particle {j}: Gamma^2 {fit[j]!r} vs {g_ref!r} (rel {rel:.2e})"
        if tc[j] != t_ref:
            assert 0 <= tc[j] < setup.n_samples, f"{context} particle {j}: tc {tc[j]} out of range"
            tie = abs(curve[tc[j]] - g_ref) / g_ref
            assert tie <= TIE_RTOL, f"{context} particle {j}: tc {tc[j]} vs {t_ref}, not a tie ({tie:.2e})"


def assert_parity_pooled(results, fit, tc, precision, context="", probe_index=0):
    """The parity rule of assert_parity on oracle_pool results: results[j] = (max Gamma^2, lowest
    argmax, [Gamma^2 at probe lags]) where probe `probe_index` is the GPU's tc of particle j."""
    for j, (g_ref, t_ref, probe) in enumerate(results):
        rel = abs(fit[j] - g_ref) / g_ref
        assert rel <= RTOL[precision], f"{context} particle {j}: Gamma^2 {fit[j]!r} vs {g_ref!r} (rel {rel:.2e})"
        if tc[j] != t_ref:
            tie = abs(probe[probe_index] - g_ref) / g_ref
            assert tie <= TIE_RTOL, f"{context} particle {j}: tc {tc[j]} vs {t_ref}, not a tie ({tie:.2e})"
