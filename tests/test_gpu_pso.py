"""GPU checks of the device lbest PSO (Sec. III) through the C ABI."""

import dataclasses
import math

import numpy as np
import pytest

import synthdata as sd
from oracle import fcas_oracle as o
from oracle import pso_oracle as po
from parity_util import RTOL, TIE_RTOL, make_ctx, oracle_setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_02150_gb300 import build as b
    b.build()


def _box(w):
    t0lo, t0hi, t15lo, t15hi = sd.chirp_time_box(w.f_low)
    return (0.0, 2 * math.pi, -0.5 * math.pi, 0.5 * math.pi, t0lo, t0hi, t15lo, t15hi)


def _cfgs(w, **kw):
    import paper_2002_02150_gb300 as fc
    return po.PsoConfig(box=_box(w), **kw), fc.pso_config(box=_box(w), **kw)


@pytest.mark.parametrize("kw", [
    dict(n_runs=3, n_particles=12, n_iter=8, seed=99, n_neighbours=1),
    dict(n_runs=2, n_particles=9, n_iter=8, seed=7, n_neighbours=2, c1=1.5, c2=2.5, vmax=0.3),
    dict(n_runs=1, n_particles=5, n_iter=10, seed=3, n_neighbours=3, w_start=0.7, w_end=0.7),   # ring wraps
    dict(n_runs=4, n_particles=16, n_iter=1, seed=12, n_neighbours=1),                          # one iteration
], ids=["default", "two-neighbours", "whole-ring", "single-iteration"])
def test_device_update_reproduces_the_oracle_step_bit_for_bit(kw):
    import torch
    import paper_2002_02150_gb300 as fc
    w = sd.SMALL
    data = sd.make_dataset(w, 0)
    setup = oracle_setup(w, data)
    ocfg, dcfg = _cfgs(w, **kw)
    n_runs, n_part = kw["n_runs"], kw["n_particles"]
    rows = n_runs * n_part
    dev = dict(device="cuda:0")
    x = torch.empty((rows, 4), dtype=torch.float64, **dev)
    v, pbx = torch.empty_like(x), torch.empty_like(x)
    pbf = torch.empty(rows, dtype=torch.float64, **dev)
    pbt = torch.empty(rows, dtype=torch.int64, **dev)
    fc.fcas_pso_init(dcfg, x, v, pbx, pbf, pbt)
    s = po.init_state(ocfg)

    def check():
        torch.cuda.synchronize()
        np.testing.assert_array_equal(x.cpu().numpy(), s.x.reshape(-1, 4))
        np.testing.assert_array_equal(v.cpu().numpy(), s.v.reshape(-1, 4))
        np.testing.assert_array_equal(pbx.cpu().numpy(), s.pbest_x.reshape(-1, 4))
        np.testing.assert_array_equal(pbf.cpu().numpy(), s.pbest_f.reshape(-1))
        np.testing.assert_array_equal(pbt.cpu().numpy(), s.pbest_tc.reshape(-1))

    check()
    outside_seen = 0
    for it in range(ocfg.n_iter):
        flat = s.x.reshape(-1, 4)
        inside = po.in_box(flat)
        outside_seen += int((~inside).sum())
        fit = np.full(rows, np.nan)        # outside the box: ignored by both sides
        tcs = np.full(rows, -1, dtype=np.int64)
        for r in np.nonzero(inside)[0]:
            fit[r], tcs[r] = o.fitness(setup, po.to_theta(ocfg, flat[r]))
        po.update(ocfg, s, it, fit.reshape(n_runs, n_part), tcs.reshape(n_runs, n_part))
        fc.fcas_pso_update(dcfg, it, torch.tensor(fit, **dev), torch.tensor(tcs, **dev), x, v, pbx, pbf, pbt)
        check()
    if ocfg.n_iter > 1:
        assert outside_seen > 0      # the let-them-fly rule was exercised


def test_search_reports_consistent_optimum():
    import torch
    import paper_2002_02150_gb300 as fc
    w = sd.SMALL
    data = sd.make_dataset(w, 1)
    _, dcfg = _cfgs(w, n_runs=2, n_particles=24, n_iter=60, seed=5)
    setup = oracle_setup(w, data)
    with make_ctx(w, data, "fp32") as ctx:
        res = fc.fcas_search(ctx, dcfg)
        assert len(res) == 2
        th = np.array([r["theta"] for r in res])
        f, t = fc.fcas_fitness(ctx, torch.tensor(th, device="cuda:0"))
        torch.cuda.synchronize()
        f, t = f.cpu().numpy(), t.cpu().numpy()
    for j, r in enumerate(res):
        assert 0 < r["evaluations"] <= 60 * 24
        assert r["fitness"] == pytest.approx(f[j], rel=1e-12) and r["tc"] == t[j]
        curve = o.fitness_curve(setup, th[j])[: setup.n_samples]
        g_ref = curve.max()
        assert abs(r["fitness"] - g_ref) / g_ref <= RTOL["fp32"]
        assert r["tc"] == int(np.argmax(curve)) or abs(curve[r["tc"]] - g_ref) / g_ref <= TIE_RTOL


def test_search_recovers_a_noiseless_injection():
    import paper_2002_02150_gb300 as fc
    w = dataclasses.replace(sd.SMALL, n_samples=sd.SMALL.n_fft)
    data = sd.make_dataset(w, 3, noise=False)
    inj = data["inj"]
    t0, _, t15, _ = o.chirp_times_from_masses(inj["m1"], inj["m2"], w.f_low)
    box = (inj["alpha"] - 0.3, inj["alpha"] + 0.3, inj["delta"] - 0.3, inj["delta"] + 0.3,
           0.97 * t0, 1.03 * t0, 0.97 * t15, 1.03 * t15)
    cfg = fc.pso_config(n_runs=4, n_particles=32, n_iter=150, seed=11, box=box)
    with make_ctx(w, data, "fp32") as ctx:
        res = fc.fcas_search(ctx, cfg)
    best = max(res, key=lambda r: r["fitness"])
    assert best["fitness"] >= 0.95 * inj["snr"] ** 2
    assert best["fitness"] <= inj["snr"] ** 2 * (1 + 1e-4)
    assert abs(best["theta"][2] / t0 - 1) < 0.01


def test_checkpoint_and_resume_is_bit_identical():
    """The swarm state is plain device arrays and the random numbers are counter based: copying the
    state to the host after 3 iterations and restoring it later continues exactly like a run that
    never stopped."""
    import torch
    import paper_2002_02150_gb300 as fc
    w = sd.SMALL
    data = sd.make_dataset(w, 2)
    _, cfg = _cfgs(w, n_runs=2, n_particles=10, n_iter=6, seed=17)
    rows = 20
    dev = dict(device="cuda:0")

    def fresh():
        x = torch.empty((rows, 4), dtype=torch.float64, **dev)
        return [x, torch.empty_like(x), torch.empty_like(x), torch.empty(rows, dtype=torch.float64, **dev),
                torch.empty(rows, dtype=torch.int64, **dev)]

    with make_ctx(w, data, "fp32") as ctx:
        def step(state, it):
            th = fc.pso_theta(cfg, state[0])
            f, t = fc.fcas_fitness(ctx, th)
            fc.fcas_pso_update(cfg, it, f, t, *state)

        a = fresh()
        fc.fcas_pso_init(cfg, *a)
        for it in range(6):
            step(a, it)
        b = fresh()
        fc.fcas_pso_init(cfg, *b)
        for it in range(3):
            step(b, it)
        saved = [t.cpu().numpy().copy() for t in b]          # checkpoint
        c = fresh()
        for dst, src in zip(c, saved):                       # resume into new buffers
            dst.copy_(torch.from_numpy(src))
        for it in range(3, 6):
            step(c, it)
        torch.cuda.synchronize()
    for u, v in zip(a, c):
        assert torch.equal(u, v)


def test_pso_run_resumes_from_a_checkpoint_file(tmp_path):
    """pso_run interrupted after 5 of 8 iterations and resumed from its last checkpoint file (written
    after iteration 4) ends exactly where an uninterrupted run ends, which is also what fcas_search
    (the same steps replayed as a graph) reports."""
    import paper_2002_02150_gb300 as fc
    w = sd.SMALL
    data = sd.make_dataset(w, 4)
    _, cfg = _cfgs(w, n_runs=2, n_particles=10, n_iter=8, seed=23)
    path = str(tmp_path / "swarm.npz")
    with make_ctx(w, data, "fp32") as ctx:
        full, n_full = fc.pso_run(ctx, cfg)
        part, n_part = fc.pso_run(ctx, cfg, checkpoint=path, every=2, stop_after=5)
        _, it, _ = fc.pso_load(path)
        resumed, n_res = fc.pso_run(ctx, cfg, checkpoint=path, every=2, resume=True)
        searched = fc.fcas_search(ctx, cfg)
        _, other = _cfgs(w, n_runs=2, n_particles=10, n_iter=8, seed=24)
        with pytest.raises(fc.FcasError):
            fc.pso_run(ctx, other, checkpoint=path, resume=True)
    assert (n_full, n_part, it, n_res) == (8, 5, 3, 8)
    for a, b, s in zip(full, resumed, searched):
        assert a == b
        assert a["fitness"] == s["fitness"] and a["tc"] == s["tc"] and a["theta"] == s["theta"]
