"""CPU checks of the C ABI: the built library exports every function include/fcas.h declares, the
binding's structs match the header's layout, and argument validation rejects bad inputs before
any device work (no compute call is made here)."""

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h")]


def _declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names.update(re.findall(r"\b(fcas_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2002_02150_gb300 import build as b
    b.build()
    import paper_2002_02150_gb300 as fc
    return fc.load_library()


def test_every_declared_function_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 8
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported by libfcas.so"


def test_struct_layouts_match_header(tmp_path):
    import paper_2002_02150_gb300.fcas as f
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "fcas.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(fcas_detector),'
                   ' sizeof(fcas_setup), offsetof(fcas_setup, fs), offsetof(fcas_setup, max_batch),'
                   ' sizeof(fcas_info), offsetof(fcas_info, sigma2), sizeof(fcas_pso_config),'
                   ' offsetof(fcas_pso_config, box), offsetof(fcas_pso_config, vmax), sizeof(fcas_search_result),'
                   ' sizeof(fcas_pso_state)); return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    expect = [ctypes.sizeof(f.fcas_detector), ctypes.sizeof(f.fcas_setup), f.fcas_setup.fs.offset,
              f.fcas_setup.max_batch.offset, ctypes.sizeof(f.fcas_info), f.fcas_info.sigma2.offset,
              ctypes.sizeof(f.fcas_pso_config), f.fcas_pso_config.box.offset, f.fcas_pso_config.vmax.offset,
              ctypes.sizeof(f.fcas_search_result), ctypes.sizeof(f.fcas_pso_state)]
    assert got == expect


def _bad_create(lib, **over):
    import paper_2002_02150_gb300.fcas as f
    s = dict(n_det=2, precision=1, n_samples=64, n_fft=64, fs=64.0, f_low=4.0, f_high=20.0, max_batch=0, flags=0)
    s.update(over)
    setup = f.fcas_setup(**s)
    dets = (f.fcas_detector * 2)()
    for d in dets:
        d.xarm[:] = [1, 0, 0]
        d.yarm[:] = [0, 1, 0]
    buf = np.zeros(4096)
    h = ctypes.c_void_p()
    rc = lib.fcas_create(ctypes.byref(h), ctypes.byref(setup), dets, buf.ctypes.data, buf.ctypes.data, None)
    return rc, lib.fcas_last_error().decode()


@pytest.mark.parametrize("over,needle", [
    (dict(n_det=0), "n_det"), (dict(n_det=9), "n_det"), (dict(precision=7), "precision"),
    (dict(n_fft=100), "power of two"), (dict(n_fft=8, n_samples=8), "power of two"),
    (dict(n_samples=65), "n_samples"), (dict(n_samples=0), "n_samples"), (dict(fs=0.0), "fs"),
    (dict(f_low=0.0), "f_low"), (dict(f_low=30.0, f_high=20.0), "f_low"), (dict(f_low=31.9, f_high=40.0), "band"),
    (dict(flags=6), "flags"),
])
def test_create_rejects_invalid_setup(lib, over, needle):
    rc, msg = _bad_create(lib, **over)
    assert rc == -1 and needle in msg


def test_null_arguments_are_rejected(lib):
    assert lib.fcas_create(None, None, None, None, None, None) == -1
    assert lib.fcas_fitness(None, 1, None, None, None, None) == -1
    assert lib.fcas_fitness_noalloc(None, 1, None, None, None, None) == -1
    assert lib.fcas_polish(None, 1, None, None, None, 1, None, 1, None, None) == -1
    assert lib.fcas_gradient(None, 1, None, None, None, None) == -1
    lib.fcas_destroy(None)
    assert lib.fcas_version() >= 100


def test_pso_config_validation(lib):
    import paper_2002_02150_gb300.fcas as f
    box = [0, 6.2, -1.5, 1.5, 1.0, 2.0, 0.1, 0.2]
    st = f.fcas_pso_state()
    for bad in (dict(n_particles=2000), dict(n_runs=0), dict(n_iter=0), dict(n_neighbours=-1)):
        kw = dict(n_runs=2, n_particles=8, n_iter=5, box=box)
        kw.update(bad)
        cfg = f.pso_config(**kw)
        assert lib.fcas_pso_init(ctypes.byref(cfg), ctypes.byref(st), None) == -1
    cfg = f.pso_config(n_runs=2, n_particles=8, n_iter=5, box=[0, 6.2, -1.5, 1.5, 2.0, 1.0, 0.1, 0.2])
    assert lib.fcas_pso_init(ctypes.byref(cfg), ctypes.byref(st), None) == -1
    assert "lo < hi" in lib.fcas_last_error().decode()
    cfg = f.pso_config(n_runs=2, n_particles=8, n_iter=5, box=box)
    assert lib.fcas_pso_init(ctypes.byref(cfg), ctypes.byref(st), None) == -1     # NULL state arrays
    assert lib.fcas_pso_update(ctypes.byref(cfg), 9, None, None, ctypes.byref(st), None) == -1
