"""Checked build (FCAS_CHECKED) of the fitness kernels: every shared-memory exchange index, stage
twiddle index and global spectrum / basis / intermediate index is recomputed from its definition
and range-tested on the device (the fast padded-address identities included); a failed test is
recorded instead of performed and makes fcas_fitness (and fcas_fitness_noalloc) return an error.
The checked library runs in a child process over every test size and compiled launch shape, and its
results (of both entry points) must equal the normal build's exactly."""

import dataclasses
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import synthdata as sd

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHECKED = os.path.join(ROOT, "paper_2002_02150_gb300", "libfcas_checked.so")

SIZES = [(16, 16, 16.0, 1.5, 6.0), (64, 50, 64.0, 5.0, 28.0), (256, 200, 128.0, 12.0, 60.0),
         (2048, 1500, 512.0, 60.0, 250.0), (16384, 12345, 1024.0, 80.0, 400.0)]

CHILD = r"""
import dataclasses, json, sys
import numpy as np
sys.path.insert(0, __ROOT__)
import synthdata as sd
import paper_2002_02150_gb300 as fc
assert fc.LIB_PATH == __LIB__, fc.LIB_PATH
cases = json.loads(sys.argv[1])
out = {}
for name, kw, precision, shapes, npart in cases:
    w = dataclasses.replace(getattr(sd, kw.pop("base")), **kw)
    data = sd.make_dataset(w, 3)
    theta = sd.make_particles(w, npart, seed=3, f_star=w.f_low)
    with fc.fcas_create(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high,
                        precision=precision) as ctx:
        for sh in shapes:
            if sh is not None:
                fc.fcas_set_shape(ctx, *sh)
            f, t = fc.fcas_fitness(ctx, theta)
            out[f"{name}/{precision}/{sh}"] = [f.tolist(), t.tolist()]
        if name.startswith("N") and shapes == [None]:
            # the allocation-free entry point of the checked library on the same particles
            import torch
            th = torch.tensor(theta, device="cuda:0")
            f2 = torch.empty(len(theta), dtype=torch.float64, device="cuda:0")
            t2 = torch.empty(len(theta), dtype=torch.int64, device="cuda:0")
            fc.fcas_fitness_noalloc(ctx, th, f2, t2)
            out[f"{name}/{precision}/noalloc"] = [f2.cpu().tolist(), t2.cpu().tolist()]
print(json.dumps(out))
"""


def _shapes(fc, w):
    ok = [None]
    with fc.fcas_create(*[sd.make_dataset(w, 3)[k] for k in ("det", "psd", "data")], w.n_fft, w.fs, w.f_low,
                        w.f_high) as ctx:
        for bias in (0, 1):
            for k in (1, 2, 4, 8, 16):
                for rb in (4, 3):
                    try:
                        fc.fcas_set_shape(ctx, bias, k, 8, rb)
                    except fc.FcasError:
                        continue
                    ok.append([bias, k, 8, rb])
    return ok


def _cases(fc):
    cases = []
    for n_fft, n_samples, fs, f_low, f_high in SIZES:
        kw = dict(base="SMALL", n_fft=n_fft, n_samples=n_samples, fs=fs, f_low=f_low, f_high=f_high,
                  arrival_s=0.3 * n_samples / fs)
        for precision in ("fp32", "fp64", "ff"):
            cases.append([f"N{n_fft}", dict(kw), precision, [None], 5])
    cases.append(["64s", dict(base="C1"), "fp32", _shapes(fc, sd.C1), 4])
    cases.append(["64s", dict(base="C1"), "fp64", [None], 3])
    cases.append(["64s", dict(base="C1"), "ff", [None], 3])
    # the 60-min transform's default shape and its one-column and radix-8 shapes
    cases.append(["60min", dict(base="C2"), "fp32", [None, [0, 1, 8, 4], [0, 2, 8, 3], [0, 4, 8, 3]], 2])
    cases.append(["60min", dict(base="C2"), "ff", [None, [0, 2, 8, 4]], 1])   # radix-8 default, radix 16
    return cases


def test_checked_build_finds_no_index_error_and_changes_no_result():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_02150_gb300 import build as b
    b.build()
    b.build(defines=["FCAS_CHECKED"], out=CHECKED)
    import paper_2002_02150_gb300 as fc
    cases = _cases(fc)
    env = dict(os.environ, FCAS_LIBRARY=CHECKED)
    child = CHILD.replace("__ROOT__", repr(ROOT)).replace("__LIB__", repr(CHECKED))
    r = subprocess.run([sys.executable, "-c", child, json.dumps(cases)], env=env, capture_output=True, text=True,
                       timeout=1800)
    assert r.returncode == 0, r.stderr[-3000:]
    got = json.loads(r.stdout.strip().splitlines()[-1])
    n = n_noalloc = 0
    for name, kw, precision, shapes, npart in cases:
        base = kw.pop("base")
        w = dataclasses.replace(getattr(sd, base), **kw)
        data = sd.make_dataset(w, 3)
        theta = sd.make_particles(w, npart, seed=3, f_star=w.f_low)
        with fc.fcas_create(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high,
                            precision=precision) as ctx:
            for sh in shapes:
                if sh is not None:
                    fc.fcas_set_shape(ctx, *sh)
                f, t = fc.fcas_fitness(ctx, theta)
                cf, ct = got[f"{name}/{precision}/{sh}"]
                assert np.array_equal(f, np.array(cf)) and np.array_equal(t, np.array(ct)), (name, precision, sh)
                n += 1
                if f"{name}/{precision}/noalloc" in got:
                    cf, ct = got[f"{name}/{precision}/noalloc"]
                    assert np.array_equal(f, np.array(cf)) and np.array_equal(t, np.array(ct)), (name, precision,
                                                                                                 "noalloc")
                    n_noalloc += 1
    assert n >= 15 and n_noalloc >= 10
