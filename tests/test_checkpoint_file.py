"""Host side of the swarm checkpoint (no GPU): the file round trip of the state and configuration,
and the binding's refusal of swarm arrays the device kernels could overrun."""

import numpy as np
import pytest

import paper_2002_02150_gb300 as fc


def _cfg(**kw):
    box = (0.0, 6.283185307179586, -1.5707963267948966, 1.5707963267948966, 1.0, 2.0, 0.1, 0.2)
    return fc.pso_config(box=box, **kw)


def test_checkpoint_round_trip(tmp_path):
    cfg = _cfg(n_runs=3, n_particles=5, n_iter=40, seed=9)
    rows = 15
    rng = np.random.default_rng(1)
    state = [rng.random((rows, 4)), rng.random((rows, 4)), rng.random((rows, 4)), rng.random(rows),
             rng.integers(0, 1 << 40, rows)]
    path = str(tmp_path / "s.npz")
    fc.pso_save(path, cfg, 17, *state)
    cfg2, it, got = fc.pso_load(path)
    assert it == 17 and bytes(cfg2) == bytes(cfg)
    for a, b in zip(state, got):
        assert a.dtype == b.dtype and np.array_equal(a, b)
    fc.pso_save(path, cfg, 18, *state)           # overwritten in place (temporary file, then rename)
    assert fc.pso_load(path)[1] == 18
    assert not (tmp_path / "s.npz.tmp.npz").exists()


def test_swarm_arrays_are_checked_before_any_launch():
    cfg = _cfg(n_runs=2, n_particles=4, n_iter=3)
    x = np.zeros((8, 4))
    with pytest.raises(fc.FcasError):             # host arrays: the kernels need device memory
        fc.fcas_pso_init(cfg, x, x, x, np.zeros(8), np.zeros(8, dtype=np.int64))
    torch = pytest.importorskip("torch")
    small = torch.zeros((7, 4), dtype=torch.float64)
    with pytest.raises(fc.FcasError):             # too few rows (and not on a GPU)
        fc.pso_theta(cfg, small, small)
