"""GPU parity of the coherent fitness (through the C ABI) against the FP64 oracle."""

import dataclasses
import math

import numpy as np
import pytest

import synthdata as sd
from oracle import fcas_oracle as o
from parity_util import RTOL, assert_parity, gpu_fitness, make_ctx, oracle_setup

pytestmark = pytest.mark.gpu

FORMS = ["fp32", "fp64", "ff"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_02150_gb300 import build as b
    b.build()


@pytest.mark.parametrize("precision", FORMS)
def test_small_workload_matches_oracle(precision):
    w = sd.SMALL
    data = sd.make_dataset(w, 0)
    theta = sd.make_particles(w, seed=0)
    with make_ctx(w, data, precision) as ctx:
        fit, tc = gpu_fitness(ctx, theta)
    assert_parity(oracle_setup(w, data), theta, fit, tc, precision, "SMALL")


# transform lengths from 2^4 to 2^14 (odd and even log2, every pass shape), ragged sample counts
SIZES = [(16, 16, 16.0, 1.5, 6.0), (32, 27, 32.0, 2.2, 12.0), (64, 50, 64.0, 5.0, 28.0),
         (128, 128, 128.0, 10.0, 50.0), (256, 200, 128.0, 12.0, 60.0), (512, 511, 256.0, 30.0, 120.0),
         (2048, 1500, 512.0, 60.0, 250.0), (8192, 8000, 512.0, 40.0, 200.0), (16384, 12345, 1024.0, 80.0, 400.0)]


@pytest.mark.parametrize("precision", FORMS)
@pytest.mark.parametrize("n_fft,n_samples,fs,f_low,f_high", SIZES)
def test_sizes_and_ragged_lengths(precision, n_fft, n_samples, fs, f_low, f_high):
    w = dataclasses.replace(sd.SMALL, n_fft=n_fft, n_samples=n_samples, fs=fs, f_low=f_low, f_high=f_high,
                            arrival_s=0.3 * n_samples / fs)
    data = sd.make_dataset(w, 3)
    theta = sd.make_particles(w, 9, seed=3, f_star=f_low)
    with make_ctx(w, data, precision) as ctx:
        fit, tc = gpu_fitness(ctx, theta)
    assert_parity(oracle_setup(w, data), theta, fit, tc, precision, f"N={n_fft}")


@pytest.mark.parametrize("precision", FORMS)
def test_noiseless_injection_gives_snr_squared(precision):
    w = dataclasses.replace(sd.SMALL, n_samples=sd.SMALL.n_fft)
    data = sd.make_dataset(w, 2, noise=False)
    inj = data["inj"]
    t0, _, t15, _ = o.chirp_times_from_masses(inj["m1"], inj["m2"], w.f_low)
    with make_ctx(w, data, precision) as ctx:
        fit, tc = gpu_fitness(ctx, [[inj["alpha"], inj["delta"], t0, t15]])
    assert fit[0] == pytest.approx(inj["snr"] ** 2, rel=RTOL[precision])
    assert tc[0] == round(inj["t_c"] * w.fs)


@pytest.mark.parametrize("precision", FORMS)
@pytest.mark.parametrize("dets", [("L1",), ("H1", "V1"), ("H1", "L1", "V1"), ("H1", "L1", "V1", "K1", "H1"),
                                  ("H1", "L1", "V1", "K1", "H1", "L1", "V1", "K1")])   # up to FCAS_MAX_DET
def test_network_sizes(precision, dets):
    w = dataclasses.replace(sd.SMALL, detectors=dets)
    data = sd.make_dataset(w, 5)
    theta = sd.make_particles(w, 6, seed=5)
    with make_ctx(w, data, precision) as ctx:
        fit, tc = gpu_fitness(ctx, theta)
    assert_parity(oracle_setup(w, data), theta, fit, tc, precision, f"D={len(dets)}")


@pytest.mark.parametrize("precision", FORMS)
def test_config1_full_batch(precision):
    w = sd.C1
    data = sd.make_dataset(w, 0)
    theta = sd.make_particles(w, seed=0)
    with make_ctx(w, data, precision) as ctx:
        fit, tc = gpu_fitness(ctx, theta)
    assert_parity(oracle_setup(w, data), theta, fit, tc, precision, "C1")


def test_chunking_and_batch_edges():
    import torch
    import paper_2002_02150_gb300 as fc
    w = sd.SMALL
    data = sd.make_dataset(w, 1)
    theta = sd.make_particles(w, 23, seed=1)
    with make_ctx(w, data, "fp32") as ref_ctx, make_ctx(w, data, "fp32", max_batch=5) as ctx:
        ref_f, ref_t = gpu_fitness(ref_ctx, theta)
        f, t = gpu_fitness(ctx, theta)
        np.testing.assert_array_equal(f, ref_f)
        np.testing.assert_array_equal(t, ref_t)
        one_f, one_t = gpu_fitness(ctx, theta[7:8])
        assert one_f[0] == ref_f[7] and one_t[0] == ref_t[7]
        # n = 0 is a no-op
        e = torch.empty((0, 4), dtype=torch.float64, device="cuda:0")
        f0, t0 = fc.fcas_fitness(ctx, e)
        assert f0.numel() == 0
        # host arrays in and out give the same numbers as device arrays
        hf, ht = fc.fcas_fitness(ctx, theta)
        np.testing.assert_array_equal(hf, ref_f)
        np.testing.assert_array_equal(ht, ref_t)


def test_invalid_particles():
    import torch
    import paper_2002_02150_gb300 as fc
    w = sd.SMALL
    data = sd.make_dataset(w, 1)
    theta = sd.make_particles(w, 4, seed=1)
    bad = theta.copy()
    bad[1, 2] = -1.0
    bad[2, 0] = math.nan
    with make_ctx(w, data, "fp32") as ctx:
        f, t = gpu_fitness(ctx, bad)
        assert np.isnan(f[1]) and t[1] == -1 and np.isnan(f[2]) and t[2] == -1
        ok_f, ok_t = gpu_fitness(ctx, theta[[0, 3]])
        assert f[0] == ok_f[0] and f[3] == ok_f[1]
        with pytest.raises(fc.FcasError):
            fc.fcas_fitness(ctx, bad)


def test_create_rejects_non_finite_inputs():
    import paper_2002_02150_gb300 as fc
    w = sd.SMALL
    data = sd.make_dataset(w, 1)
    d = data["data"].copy()
    d[2, 17] = math.inf
    with pytest.raises(fc.FcasError, match="non-finite"):
        fc.fcas_create(data["det"], data["psd"], d, w.n_fft, w.fs, w.f_low, w.f_high)
    p = data["psd"].copy()
    p[0, 700] = 0.0          # inside the band (640, 2000] of this workload
    with pytest.raises(fc.FcasError, match="psd"):
        fc.fcas_create(data["det"], p, data["data"], w.n_fft, w.fs, w.f_low, w.f_high)


def test_profiling_counts_launches():
    import paper_2002_02150_gb300 as fc
    w = sd.SMALL
    data = sd.make_dataset(w, 1)
    theta = sd.make_particles(w, 10, seed=1)
    with make_ctx(w, data, "fp32", max_batch=4) as ctx:
        fc.fcas_profile_enable(ctx, True)
        gpu_fitness(ctx, theta)
        ms, n = fc.fcas_profile_read(ctx, "pass_a")
        assert n == 3 and ms > 0
        assert fc.fcas_profile_read(ctx, "geometry")[1] == 1
        info = fc.fcas_get_info(ctx)
        assert info["n1"] * info["n2"] == w.n_fft and info["chunk"] == 4


def test_config2_full_size_sampled():
    """The 60-min workload in the launch configuration the benchmark times (320 particles in chunks
    of 64): every particle has a finite, non-negative fitness and an in-range tc; 32 particles spread
    over every chunk match the oracle one by one in the FP32 and float-float forms, and 8 of them in
    the binary64 form (the oracle runs on the host cores, one process per particle at a time)."""
    from oracle_pool import oracle_curves
    from parity_util import assert_parity_pooled
    w = sd.C2
    data = sd.make_dataset(w, 0)
    theta = sd.make_particles(w, seed=0)
    sample = np.linspace(0, len(theta) - 1, 32).astype(int)
    sample64 = sample[::4]
    got = {}
    for precision in FORMS:
        with make_ctx(w, data, precision) as ctx:
            fit, tc = gpu_fitness(ctx, theta if precision == "fp32" else theta[sample if precision == "ff" else sample64])
        if precision == "fp32":
            assert np.all(np.isfinite(fit)) and np.all(fit >= 0)
            assert np.all((tc >= 0) & (tc < w.n_samples))
            fit, tc = fit[sample], tc[sample]
        got[precision] = (fit, tc)
    del data
    probes = [[got["fp32"][1][j], got["ff"][1][j]] + ([got["fp64"][1][j // 4]] if j % 4 == 0 else [])
              for j in range(len(sample))]
    ref = oracle_curves(w, 0, theta[sample], probes)
    assert_parity_pooled(ref, *got["fp32"], "fp32", "C2 fp32", probe_index=0)
    assert_parity_pooled(ref, *got["ff"], "ff", "C2 ff", probe_index=1)
    assert_parity_pooled(ref[::4], *got["fp64"], "fp64", "C2 fp64", probe_index=2)


def test_largest_supported_length_sampled():
    """N = 2^24 (the largest transform the two passes cover: 2^12 x 2^12), a ragged data length
    and a two-detector network; the first particles match the oracle one by one in the FP32 and
    float-float forms."""
    w = dataclasses.replace(sd.C2, detectors=("H1", "L1"), n_fft=1 << 24, n_samples=(1 << 24) - 12345, fs=4096.0,
                            f_low=30.0, f_high=1500.0, arrival_s=2000.0, n_particles=6)
    data = sd.make_dataset(w, 7)
    theta = sd.make_particles(w, seed=7)
    setup = oracle_setup(w, data)
    for precision in ("fp32", "ff"):
        with make_ctx(w, data, precision) as ctx:
            fit, tc = gpu_fitness(ctx, theta)
        assert np.all(np.isfinite(fit)) and np.all((tc >= 0) & (tc < w.n_samples))
        assert_parity(setup, theta[:2], fit[:2], tc[:2], precision, f"N=2^24 {precision}")


def test_two_contexts_on_two_streams_match_sequential_results():
    """Contexts hold no shared state: calls on two streams overlapping on the GPU give the results
    of the same calls made one after the other."""
    import torch
    import paper_2002_02150_gb300 as fc
    w = sd.C1
    d1, d2 = sd.make_dataset(w, 51), sd.make_dataset(w, 52)
    th = torch.tensor(sd.make_particles(w, 96, seed=51), device="cuda:0")
    with make_ctx(w, d1, "fp32") as c1, make_ctx(w, d2, "fp32") as c2:
        ref1 = [x.clone() for x in fc.fcas_fitness(c1, th)]
        ref2 = [x.clone() for x in fc.fcas_fitness(c2, th)]
        torch.cuda.synchronize()
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        outs = []
        for _ in range(4):
            f1 = torch.empty(96, dtype=torch.float64, device="cuda:0")
            t1 = torch.empty(96, dtype=torch.int64, device="cuda:0")
            f2, t2 = torch.empty_like(f1), torch.empty_like(t1)
            fc.fcas_fitness(c1, th, f1, t1, stream=s1.cuda_stream)
            fc.fcas_fitness(c2, th, f2, t2, stream=s2.cuda_stream)
            outs.append((f1, t1, f2, t2))
        torch.cuda.synchronize()
    for f1, t1, f2, t2 in outs:
        assert torch.equal(f1, ref1[0]) and torch.equal(t1, ref1[1])
        assert torch.equal(f2, ref2[0]) and torch.equal(t2, ref2[1])


def test_condition_number_matches_the_oracle():
    import torch
    import paper_2002_02150_gb300 as fc
    w = sd.SMALL
    data = sd.make_dataset(w, 61)
    theta = sd.make_particles(w, 200, seed=61)
    theta[:2, :2] = [[math.radians(32.09), math.radians(-53.86)], [math.radians(150.11), math.radians(-60.16)]]
    with make_ctx(w, data, "fp32") as ctx:
        k_host = fc.fcas_condition_number(ctx, theta)
        k_dev = fc.fcas_condition_number(ctx, torch.tensor(theta, device="cuda:0")).cpu().numpy()
    ref = np.array([o.condition_number(np.asarray(data["det"]), th[0], th[1]) for th in theta])
    np.testing.assert_allclose(k_host, ref, rtol=1e-10)
    assert np.array_equal(k_host, k_dev)
    # one detector: rank one everywhere
    w1 = dataclasses.replace(sd.SMALL, detectors=("L1",))
    d1 = sd.make_dataset(w1, 62)
    with make_ctx(w1, d1, "fp64") as ctx1:
        assert np.all(np.isinf(fc.fcas_condition_number(ctx1, theta[:10])))


@pytest.mark.parametrize("precision", FORMS)
def test_paper_chirp_time_box_at_f_star_10hz(precision):
    """The paper's search box at f_* = 10 Hz (Sec. V: tau0 up to 1500 s, chirp phases of up to
    ~10^4 turns at the low-frequency end), on a 512-s segment at 512 Hz, band 10-200 Hz."""
    w = dataclasses.replace(sd.PAPER_DNS, fs=512.0, n_samples=250000, n_fft=1 << 18, f_high=200.0, arrival_s=20.0)
    data = sd.make_dataset(w, 71)
    lo0, hi0, lo15, hi15 = sd.PAPER_TAU_BOX
    rng = np.random.default_rng(71)
    theta = np.stack([rng.uniform(0, 2 * math.pi, 6), np.arcsin(rng.uniform(-1, 1, 6)),
                      rng.uniform(lo0, hi0, 6), rng.uniform(lo15, hi15, 6)], axis=1)
    with make_ctx(w, data, precision) as ctx:
        fit, tc = gpu_fitness(ctx, theta)
    assert_parity(oracle_setup(w, data), theta, fit, tc, precision, "f*=10Hz")


def _split_log_n1(log_n):
    """log2 of the pass-B length N1 the library uses for a length-2^log_n transform (N = N1 N2 with
    N2 = 2^max(2, log_n - 13, floor(log_n / 2)))."""
    return log_n - max(2, log_n - 13, log_n // 2)


@pytest.mark.parametrize("precision", FORMS)
@pytest.mark.parametrize("log_n", [14, 15])
def test_exact_ties_resolve_to_the_lowest_lag(precision, log_n):
    """Data with period P = N1 (the create-time transform's first length) has a spectrum that is
    exactly zero off the multiples of N / P in every step of the library (transforms of constant
    columns, zeros times twiddles), so Gamma^2(t) repeats exactly with period P and every maximum is
    tied with its copies P, 2P, ... later. The library must return the lowest of the tied lags, as
    np.argmax does: tc < P, on the oracle's maximum modulo P (or a tie within 1e-5)."""
    import paper_2002_02150_gb300 as fc
    n = 1 << log_n
    period = 1 << _split_log_n1(log_n)
    w = dataclasses.replace(sd.SMALL, n_fft=n, n_samples=n, fs=1024.0, f_low=40.0, f_high=200.0)
    base = sd.make_dataset(w, 81, inject=False)
    rng = np.random.default_rng(81)
    data = np.tile(rng.standard_normal((w.n_det, period)) * 1e-21, (1, n // period))
    theta = sd.make_particles(w, 6, seed=81)
    with fc.fcas_create(base["det"], base["psd"], data, w.n_fft, w.fs, w.f_low, w.f_high, precision=precision) as ctx:
        assert fc.fcas_get_info(ctx)["n1"] == period
        fit, tc = gpu_fitness(ctx, theta)
    setup = o.OracleSetup(base["det"], base["psd"], data, w.n_fft, w.fs, w.f_low, w.f_high)
    for j, th in enumerate(theta):
        curve = o.fitness_curve(setup, th)
        # the premise: the oracle's curve repeats with period P (to its own rounding)
        assert np.max(np.abs(curve - np.tile(curve[:period], n // period))) <= 1e-9 * curve.max()
        g_ref = curve.max()
        assert abs(fit[j] - g_ref) / g_ref <= RTOL[precision]
        assert 0 <= tc[j] < period, f"particle {j}: tc {tc[j]} is not the lowest of the tied lags"
        t_ref = int(np.argmax(curve[:period]))
        if tc[j] != t_ref:
            assert abs(curve[tc[j]] - g_ref) / g_ref <= 1e-5, (j, tc[j], t_ref)


@pytest.mark.parametrize("precision", FORMS)
def test_zero_data_ties_every_lag_at_zero(precision):
    """All-zero data: Gamma^2(t) = 0 for every lag, so the maximum is 0 and the lowest lag is 0."""
    import paper_2002_02150_gb300 as fc
    w = sd.SMALL
    base = sd.make_dataset(w, 82, inject=False)
    theta = sd.make_particles(w, 5, seed=82)
    with fc.fcas_create(base["det"], base["psd"], np.zeros((w.n_det, w.n_samples)), w.n_fft, w.fs, w.f_low,
                        w.f_high, precision=precision) as ctx:
        fit, tc = gpu_fitness(ctx, theta)
    np.testing.assert_array_equal(fit, np.zeros(5))
    np.testing.assert_array_equal(tc, np.zeros(5, dtype=np.int64))


@pytest.mark.parametrize("precision", FORMS)
def test_null_psd_is_the_analytic_aligo_fit(precision):
    """psd = NULL at create evaluates the analytic aLIGO fit on the device: the context equals one
    created from the same fit sampled on the host (to the rounding of the two evaluations of the fit)
    and matches the oracle given the host-sampled fit."""
    import paper_2002_02150_gb300 as fc
    w = sd.C1
    data = sd.make_dataset(w, 83)
    theta = sd.make_particles(w, 12, seed=83)
    with fc.fcas_create(data["det"], None, data["data"], w.n_fft, w.fs, w.f_low, w.f_high, precision=precision) as c0, \
            make_ctx(w, data, precision) as c1:
        i0, i1 = fc.fcas_get_info(c0), fc.fcas_get_info(c1)
        np.testing.assert_allclose(i0["sigma2"][:w.n_det], i1["sigma2"][:w.n_det], rtol=1e-13)
        f0, t0 = gpu_fitness(c0, theta)
        f1, t1 = gpu_fitness(c1, theta)
    np.testing.assert_allclose(f0, f1, rtol=1e-6 if precision == "fp32" else 1e-12)
    np.testing.assert_array_equal(t0, t1)
    assert_parity(oracle_setup(w, data), theta, f0, t0, precision, "psd=NULL")


@pytest.mark.parametrize("k1b,radix_bits,f_low,cmax", [(4, 4, 42.0, 3), (4, 3, 42.0, 3), (8, 4, 90.0, 7)])
def test_shared_chirp_phase_and_its_per_particle_fallback(k1b, radix_bits, f_low, cmax):
    """FP32 pass A with four (eight) columns per CTA steps the chirp phase of adjacent bins from
    anchor bins only for particles whose remainder bound for steps of up to 3 (7) bins is below 1e-7
    turns, and forms every bin itself for the others. A 128-s segment whose band starts at 42 Hz
    (90 Hz) puts the bound's threshold inside the chirp-time box: the particles at the box's lowest
    tau0 qualify, those above do not. One launch holds both kinds, each checked against the oracle."""
    import paper_2002_02150_gb300 as fc
    from test_taylor_bound import bound, coefficients
    w = dataclasses.replace(sd.C1, name="4det-128s-8192Hz", fs=8192.0, n_fft=1 << 20, n_samples=(1 << 20) - 4321,
                            f_low=f_low, f_high=400.0, arrival_s=40.0)
    data = sd.make_dataset(w, 11)
    rng = np.random.default_rng(11)
    t0lo, t0hi, t15lo, t15hi = sd.chirp_time_box(w.f_low)
    span = (t0hi - t0lo) / 36.0   # 1 s at 42 Hz
    tau0 = np.concatenate([np.linspace(t0lo, t0lo + 0.25 * span, 5), np.linspace(t0lo + 2.0 * span, t0hi, 5)])
    tau15 = rng.uniform(t15lo, t15hi, tau0.size)
    theta = np.stack([rng.uniform(0, 2 * np.pi, tau0.size), np.arcsin(rng.uniform(-1, 1, tau0.size)), tau0, tau15], 1)
    df = w.fs / w.n_fft
    shared = [bound(coefficients(a, b, w.f_low), w.f_low, df, cmax) < 1e-7 for a, b in zip(tau0, tau15)]
    assert any(shared) and not all(shared), shared
    with make_ctx(w, data, "fp32") as ctx:
        info = fc.fcas_set_shape(ctx, 0, k1b, 8, radix_bits)
        assert info["k1b"] == k1b and info["radix_bits_a"] == radix_bits
        fit, tc = gpu_fitness(ctx, theta)
    assert_parity(oracle_setup(w, data), theta, fit, tc, "fp32", f"shared chirp phase, K1B {k1b}, radix bits {radix_bits}")
