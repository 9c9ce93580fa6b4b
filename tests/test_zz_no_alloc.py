"""fcas_fitness_noalloc, the allocation-free entry point, through the C ABI.

The allocation-free call exists for programs that may not allocate device memory once they run
(memory owned by another runtime's pool, or a footprint fixed at start-up); its scratch is a fixed
static device array inside the library. Checked here: its results against fcas_fitness and against
the FP64 oracle, two calls in a row (the array is shared and keeps the previous call's contents),
chunking, that calls after the set-up call leave the device's free memory and torch's allocations
unchanged, and its rejections. This file is collected last so that a failure here never hides
another test, and it passes both alone in a fresh process and after the rest of the suite.
"""

import dataclasses

import numpy as np
import pytest

import synthdata as sd
from parity_util import RTOL, assert_parity, make_ctx, oracle_setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_02150_gb300 import build as b
    b.build()


def _compare(w, precision, n, oracle=False):
    import torch
    import paper_2002_02150_gb300 as fc
    data = sd.make_dataset(w, 4)
    theta_h = sd.make_particles(w, n, seed=4)
    theta = torch.tensor(theta_h, device="cuda:0")
    with make_ctx(w, data, precision) as ctx:
        ref_f, ref_t = fc.fcas_fitness(ctx, theta)
        for _ in range(2):                      # two calls in a row share (and reuse) the static scratch
            f = torch.full((n,), -7.0, dtype=torch.float64, device="cuda:0")
            t = torch.full((n,), -7, dtype=torch.int64, device="cuda:0")
            fc.fcas_fitness_noalloc(ctx, theta, f, t)
            torch.cuda.synchronize()
            np.testing.assert_allclose(f.cpu().numpy(), ref_f.cpu().numpy(), rtol=RTOL[precision], atol=0)
            np.testing.assert_array_equal(t.cpu().numpy(), ref_t.cpu().numpy())
            if oracle:
                assert_parity(oracle_setup(w, data), theta_h, f.cpu().numpy(), t.cpu().numpy(), precision,
                              f"noalloc {w.name} {precision}")


@pytest.mark.parametrize("precision", ["fp32", "fp64", "ff"])
def test_noalloc_matches_fitness_and_oracle_small(precision):
    _compare(sd.SMALL, precision, 37, oracle=True)


def test_noalloc_matches_fitness_and_oracle_64s_segment_in_chunks():
    # 2^16 points in FP32 need 1 MiB of scratch per particle: 40 particles take two chunks
    _compare(sd.C1, "fp32", 40, oracle=True)


def test_noalloc_allocates_nothing_after_the_setup_call():
    """After one set-up call per context (which loads the library's no-alloc module on the device and
    every kernel the calls use), further calls of several batch sizes and forms leave the device's free
    memory (cudaMemGetInfo) and torch's allocated bytes exactly as they were."""
    import torch
    import paper_2002_02150_gb300 as fc
    cases = []
    for w, precision in ((sd.SMALL, "fp32"), (sd.SMALL, "fp64"), (sd.SMALL, "ff"), (sd.C1, "fp32")):
        data = sd.make_dataset(w, 5)
        theta = torch.tensor(sd.make_particles(w, 64, seed=5), device="cuda:0")
        cases.append((make_ctx(w, data, precision), theta))
    outs = {n: (torch.empty(n, dtype=torch.float64, device="cuda:0"), torch.empty(n, dtype=torch.int64, device="cuda:0"))
            for n in (1, 7, 64)}
    try:
        for ctx, theta in cases:                           # set-up calls
            for n, (f, t) in outs.items():
                fc.fcas_fitness_noalloc(ctx, theta[:n], f, t)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        alloc0 = torch.cuda.memory_allocated()
        for _ in range(3):
            for ctx, theta in cases:
                for n, (f, t) in outs.items():
                    fc.fcas_fitness_noalloc(ctx, theta[:n], f, t)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
        assert torch.cuda.memory_allocated() == alloc0
    finally:
        for ctx, _ in cases:
            ctx.close()


def test_noalloc_rejects_oversized_segment_and_host_arrays():
    import torch
    import paper_2002_02150_gb300 as fc
    w = dataclasses.replace(sd.SMALL, n_fft=1 << 21, n_samples=1 << 21, fs=4096.0, f_low=100.0, f_high=300.0)
    data = sd.make_dataset(w, 1, inject=False)
    theta = torch.tensor(sd.make_particles(w, 2, seed=1), device="cuda:0")
    f = torch.empty(2, dtype=torch.float64, device="cuda:0")
    t = torch.empty(2, dtype=torch.int64, device="cuda:0")
    with make_ctx(w, data, "fp32") as ctx:
        with pytest.raises(fc.FcasError, match="static scratch holds"):
            fc.fcas_fitness_noalloc(ctx, theta, f, t)
    with make_ctx(sd.SMALL, sd.make_dataset(sd.SMALL, 1), "fp32") as ctx:
        lib = fc.load_library()
        th_h = np.zeros((2, 4))
        rc = lib.fcas_fitness_noalloc(ctx.handle, 2, th_h.ctypes.data, f.data_ptr(), t.data_ptr(), None)
        assert rc == -1 and "device memory" in fc.fcas_last_error()
        with pytest.raises(ValueError, match="need 2 elements"):
            fc.fcas_fitness_noalloc(ctx, theta, f[:1], t)
        with pytest.raises(ValueError, match="shape"):
            fc.fcas_fitness_noalloc(ctx, theta.reshape(-1), f, t)
