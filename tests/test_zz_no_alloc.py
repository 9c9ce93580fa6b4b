"""fcas_fitness_noalloc, the allocation-free entry point, against fcas_fitness (through the C ABI).

The allocation-free call exists for programs that may not allocate device memory once they run
(memory owned by another runtime's pool, or a footprint fixed at start-up); its scratch is a fixed
static device array inside the library. This file is collected last so that a failure here never
hides another test, and it passes both alone in a fresh process and after the rest of the suite.
"""

import dataclasses

import numpy as np
import pytest

import synthdata as sd
from parity_util import RTOL, make_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_02150_gb300 import build as b
    b.build()


def _compare(w, precision, n):
    import torch
    import paper_2002_02150_gb300 as fc
    data = sd.make_dataset(w, 4)
    theta = torch.tensor(sd.make_particles(w, n, seed=4), device="cuda:0")
    with make_ctx(w, data, precision) as ctx:
        ref_f, ref_t = fc.fcas_fitness(ctx, theta)
        for _ in range(2):                      # two calls in a row share (and reuse) the static scratch
            f = torch.full((n,), -7.0, dtype=torch.float64, device="cuda:0")
            t = torch.full((n,), -7, dtype=torch.int64, device="cuda:0")
            fc.fcas_fitness_noalloc(ctx, theta, f, t)
            torch.cuda.synchronize()
            np.testing.assert_allclose(f.cpu().numpy(), ref_f.cpu().numpy(), rtol=RTOL[precision], atol=0)
            np.testing.assert_array_equal(t.cpu().numpy(), ref_t.cpu().numpy())


@pytest.mark.parametrize("precision", ["fp32", "fp64", "ff"])
def test_noalloc_matches_fitness_small(precision):
    _compare(sd.SMALL, precision, 37)


def test_noalloc_matches_fitness_64s_segment_in_chunks():
    # 2^16 points in FP32 need 1 MiB of scratch per particle: 40 particles take two chunks
    _compare(sd.C1, "fp32", 40)


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
        assert rc == -1 and "device pointers" in fc.fcas_last_error()
