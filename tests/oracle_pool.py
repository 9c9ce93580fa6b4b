"""The FP64 oracle over many particles of one workload on the host cores: spawned worker processes
(never forked from a process that has used the GPU), each preparing its own oracle setup of the
seeded data once and then evaluating whole fitness curves one particle at a time."""

import dataclasses
import multiprocessing as mp
import os

import numpy as np

_setup = None


def _mem_available_bytes():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return None


def _init(wname, overrides, seed):
    global _setup
    import synthdata as sd
    from oracle import fcas_oracle as o
    w = dataclasses.replace(sd.workload_by_name(wname), **overrides)
    data = sd.make_dataset(w, seed)
    _setup = o.OracleSetup(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high)


def _eval(args):
    """(max over t < n_samples of Gamma^2(t), its lowest argmax, Gamma^2 at each probe lag)."""
    from oracle import fcas_oracle as o
    theta, probes = args
    curve = o.fitness_curve(_setup, np.asarray(theta))[: _setup.n_samples]
    t = int(np.argmax(curve))
    return float(curve[t]), t, [float(curve[p]) if 0 <= p < len(curve) else float("nan") for p in probes]


def oracle_curves(w, seed, thetas, probes, base=None, overrides=None):
    """Oracle results for each particle of `thetas` on workload `w` (a synthdata workload, or the
    named workload `base` with the fields `overrides` replaced) with data seed `seed`; `probes[j]`
    lists the lags whose Gamma^2 is returned for particle j. Worker count: the host cores, bounded
    by the memory one worker needs."""
    name = base or w.name
    per_worker = 3.0e9 if w.n_fft >= 1 << 22 else 0.5e9
    n = min(os.cpu_count() or 1, len(thetas))
    avail = _mem_available_bytes()
    if avail:
        n = max(1, min(n, int(avail * 0.6 // per_worker)))
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(n, initializer=_init, initargs=(name, dict(overrides or {}), seed)) as pool:
            return pool.map(_eval, [(list(map(float, th)), list(map(int, pr))) for th, pr in zip(thetas, probes)],
                            chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
