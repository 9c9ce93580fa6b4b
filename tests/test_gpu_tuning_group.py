"""Launch shapes (every compiled variant keeps parity), the autotuner and its cache, and group
searches over segments of different lengths (identical to the individual searches)."""

import dataclasses
import math

import numpy as np
import pytest

import synthdata as sd
from parity_util import assert_parity, gpu_fitness, make_ctx, oracle_setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_02150_gb300 import build as b
    b.build()


def _shapes(ctx):
    import paper_2002_02150_gb300 as fc
    out = []
    for bias in (0, 1):
        for k in (1, 2, 4, 8, 16):
            for rb in (4, 3):
                try:
                    fc.fcas_set_shape(ctx, bias, k, 8, rb)
                except fc.FcasError:
                    continue
                for sub in (1, 8):
                    out.append((bias, k, sub, rb))
    return out


@pytest.mark.parametrize("w", [sd.SMALL, sd.C1], ids=["small", "64s"])
def test_every_compiled_shape_matches_the_oracle(w):
    import paper_2002_02150_gb300 as fc
    data = sd.make_dataset(w, 6)
    theta = sd.make_particles(w, 6, seed=6)
    setup = oracle_setup(w, data)
    with make_ctx(w, data, "fp32") as ctx:
        shapes = _shapes(ctx)
        assert len(shapes) >= 4
        for bias, k, sub, rb in shapes:
            info = fc.fcas_set_shape(ctx, bias, k, sub, rb)
            assert (info["split_bias"], info["k1b"], info["sub"], info["radix_bits_a"]) == (bias, k, sub, rb)
            assert info["n1"] * info["n2"] == w.n_fft
            f, t = gpu_fitness(ctx, theta)
            assert_parity(setup, theta, f, t, "fp32", f"shape {bias, k, sub, rb}")


def test_shapes_of_the_60min_transform_agree():
    import paper_2002_02150_gb300 as fc
    w = sd.C2
    data = sd.make_dataset(w, 0)
    theta = sd.make_particles(w, 6, seed=2)
    with make_ctx(w, data, "fp32", max_batch=8) as ctx:
        ref_f, ref_t = gpu_fitness(ctx, theta)
        shapes = _shapes(ctx)
        assert len(shapes) >= 4 and any(rb == 3 for *_, rb in shapes)
        for bias, k, sub, rb in shapes:
            fc.fcas_set_shape(ctx, bias, k, sub, rb)
            f, t = gpu_fitness(ctx, theta)
            np.testing.assert_allclose(f, ref_f, rtol=2e-5)
            np.testing.assert_array_equal(t, ref_t)


def test_autotune_applies_the_fastest_shape_and_caches_it(tmp_path):
    import paper_2002_02150_gb300 as fc
    w = sd.C1
    data = sd.make_dataset(w, 1)
    cache = str(tmp_path / "tune.txt")
    theta = sd.make_particles(w, 8, seed=1)
    with make_ctx(w, data, "fp32") as ctx:
        info = fc.fcas_autotune(ctx, 64, cache)
        assert info["tuned_ms_per_particle"] > 0
        f, t = gpu_fitness(ctx, theta)
        assert_parity(oracle_setup(w, data), theta, f, t, "fp32", "tuned")
    lines = open(cache).read().splitlines()
    assert len(lines) == 1
    with make_ctx(w, data, "fp32") as ctx2:
        info2 = fc.fcas_autotune(ctx2, 64, cache)
        for key in ("split_bias", "k1b", "sub", "radix_bits_a"):
            assert info2[key] == info[key]
    assert len(open(cache).read().splitlines()) == 1      # a hit adds nothing


def test_group_search_equals_individual_searches():
    import paper_2002_02150_gb300 as fc
    base = sd.SMALL
    segs = [dataclasses.replace(base, n_fft=2048, n_samples=2000),
            dataclasses.replace(base, n_fft=4096, n_samples=3600),
            dataclasses.replace(base, n_fft=8192, n_samples=8192)]
    datas = [sd.make_dataset(w, 20 + s) for s, w in enumerate(segs)]
    t0lo, t0hi, t15lo, t15hi = sd.chirp_time_box(base.f_low)
    box = (0.0, 2 * math.pi, -0.5 * math.pi, 0.5 * math.pi, t0lo, t0hi, t15lo, t15hi)
    cfg = fc.pso_config(n_runs=2, n_particles=16, n_iter=30, seed=5, box=box)
    ctxs = [fc.fcas_create(d["det"], d["psd"], d["data"], w.n_fft, w.fs, w.f_low, w.f_high,
                           flags=fc.FCAS_SETUP_LAZY_SCRATCH) for w, d in zip(segs, datas)]
    with fc.fcas_group_create(ctxs, max_batch=7) as grp:
        got = grp.search(cfg)
    for s, ctx in enumerate(ctxs):
        ref = fc.fcas_search(ctx, fc.pso_config(n_runs=2, n_particles=16, n_iter=30, seed=fc.segment_seed(5, s),
                                                box=box))
        assert got[s] == ref
        ctx.close()


def test_group_of_mixed_precisions_equals_individual_searches():
    import paper_2002_02150_gb300 as fc
    base = sd.SMALL
    segs = [(base, "fp32"), (base, "fp64"), (dataclasses.replace(base, n_fft=8192, n_samples=6000), "ff")]
    t0lo, t0hi, t15lo, t15hi = sd.chirp_time_box(base.f_low)
    box = (0.0, 2 * math.pi, -0.5 * math.pi, 0.5 * math.pi, t0lo, t0hi, t15lo, t15hi)
    cfg = fc.pso_config(n_runs=2, n_particles=8, n_iter=12, seed=11, box=box)
    ctxs = []
    for s, (w, prec) in enumerate(segs):
        d = sd.make_dataset(w, 40 + s)
        ctxs.append(fc.fcas_create(d["det"], d["psd"], d["data"], w.n_fft, w.fs, w.f_low, w.f_high, precision=prec,
                                   flags=fc.FCAS_SETUP_LAZY_SCRATCH))
    with fc.fcas_group_create(ctxs, max_batch=5) as grp:
        got = grp.search(cfg)
    for s, ctx in enumerate(ctxs):
        ref = fc.fcas_search(ctx, fc.pso_config(n_runs=2, n_particles=8, n_iter=12, seed=fc.segment_seed(11, s),
                                                box=box))
        assert got[s] == ref
        ctx.close()


def test_float_float_radix8_shape_on_the_60min_transform():
    """The float-float form's radix-8 pass A (512-thread CTAs of two 2048-point columns) against its
    radix-16 pass A and the oracle."""
    import paper_2002_02150_gb300 as fc
    w = sd.C2
    data = sd.make_dataset(w, 0)
    theta = sd.make_particles(w, 4, seed=3)
    with make_ctx(w, data, "ff", max_batch=4) as ctx:
        info = fc.fcas_set_shape(ctx, 0, 2, 8, 4)
        assert info["n2"] == 2048
        ref_f, ref_t = gpu_fitness(ctx, theta)
        info = fc.fcas_set_shape(ctx, 0, 2, 8, 3)
        assert info["radix_bits_a"] == 3
        f, t = gpu_fitness(ctx, theta)
    np.testing.assert_allclose(f, ref_f, rtol=1e-12)
    np.testing.assert_array_equal(t, ref_t)
    assert_parity(oracle_setup(w, data), theta[:2], f[:2], t[:2], "ff", "radix-8 float-float")
