"""Background and chirp-time tiling rows: time-shifted contexts (Sec. V time shifts) and groups
searching one segment over several (tau0, tau1.5) rectangles (Sec. IV)."""

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


def _rolled(data, shifts):
    out = dict(data)
    out["data"] = np.stack([np.roll(np.asarray(x), int(s)) for x, s in zip(data["data"], shifts)])
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp64", "ff"])
def test_time_shifted_context_equals_a_context_of_the_rolled_data(precision):
    import paper_2002_02150_gb300 as fc
    w = sd.SMALL
    data = sd.make_dataset(w, 31)
    theta = sd.make_particles(w, 12, seed=31)
    shifts = [0, 7, -5, w.n_samples + 3]            # negative and beyond n_samples: taken mod n_samples
    rolled = _rolled(data, shifts)
    with fc.fcas_create(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high,
                        precision=precision, shifts=shifts) as a, make_ctx(w, rolled, precision) as b:
        fa, ta = gpu_fitness(a, theta)
        fb, tb = gpu_fitness(b, theta)
    assert np.array_equal(fa, fb) and np.array_equal(ta, tb)
    # and the oracle on the rolled series (the shift is input preparation: x'_i[t] = x_i[t - s_i])
    assert_parity(oracle_setup(w, rolled), theta, fa, ta, precision, "time-shifted")


def test_time_shift_leaves_the_callers_device_data_untouched():
    import torch
    import paper_2002_02150_gb300 as fc
    w = sd.SMALL
    data = sd.make_dataset(w, 32)
    dev = torch.tensor(np.asarray(data["data"]), device="cuda:0")
    before = dev.clone()
    with fc.fcas_create(data["det"], data["psd"], dev, w.n_fft, w.fs, w.f_low, w.f_high, shifts=[1, 2, 3, 4]):
        torch.cuda.synchronize()
    assert torch.equal(dev, before)


def test_tiled_group_search_equals_one_search_per_tile():
    import paper_2002_02150_gb300 as fc
    w = sd.SMALL
    data = sd.make_dataset(w, 33)
    t0lo, t0hi, t15lo, t15hi = sd.chirp_time_box(w.f_low)
    boxes = fc.fcas_tau_tiles(t0lo, t0hi, t15lo, t15hi, 2, 2, 0.1)
    cfg = fc.pso_config(n_runs=2, n_particles=12, n_iter=25, seed=9, box=tuple(boxes[0]))
    ctx = fc.fcas_create(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high,
                         flags=fc.FCAS_SETUP_LAZY_SCRATCH)
    with fc.fcas_group_create([ctx] * len(boxes), max_batch=5) as grp:
        got = grp.search(cfg, boxes=boxes)
    for s, box in enumerate(boxes):
        ref = fc.fcas_search(ctx, fc.pso_config(n_runs=2, n_particles=12, n_iter=25, seed=fc.segment_seed(9, s),
                                                box=tuple(box)))
        assert got[s] == ref
        for r in got[s]:                       # every reported optimum lies in its own tile
            assert box[4] <= r["theta"][2] <= box[5] and box[6] <= r["theta"][3] <= box[7]
    ctx.close()


def test_an_invalid_tile_box_names_its_segment():
    import paper_2002_02150_gb300 as fc
    w = sd.SMALL
    data = sd.make_dataset(w, 34)
    t0lo, t0hi, t15lo, t15hi = sd.chirp_time_box(w.f_low)
    boxes = fc.fcas_tau_tiles(t0lo, t0hi, t15lo, t15hi, 1, 2, 0.0)
    boxes[1, 4], boxes[1, 5] = boxes[1, 5], boxes[1, 4]          # lo > hi in segment 1
    cfg = fc.pso_config(n_runs=1, n_particles=4, n_iter=2, seed=1, box=tuple(boxes[0]))
    ctx = fc.fcas_create(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high)
    with fc.fcas_group_create([ctx, ctx], max_batch=4) as grp:
        with pytest.raises(fc.FcasError, match="segment 1"):
            grp.search(cfg, boxes=boxes)
    ctx.close()


def test_tiled_search_finds_the_injection_in_its_tile():
    import paper_2002_02150_gb300 as fc
    w = sd.C1
    data = sd.make_dataset(w, 0, inject=True, snr=12.0)
    inj = data["inj"]
    from oracle import fcas_oracle as o
    tau0_inj = o.chirp_times_from_masses(inj["m1"], inj["m2"], w.f_low)[0]
    t0lo, t0hi, t15lo, t15hi = sd.chirp_time_box(w.f_low)
    boxes = fc.fcas_tau_tiles(t0lo, t0hi, t15lo, t15hi, 2, 1, 0.2)
    cfg = fc.pso_config(n_runs=4, n_particles=40, n_iter=1000, seed=3, box=tuple(boxes[0]))
    ctx = fc.fcas_create(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high,
                         flags=fc.FCAS_SETUP_LAZY_SCRATCH)
    with fc.fcas_group_create([ctx] * len(boxes)) as grp:
        res = grp.search(cfg, boxes=boxes)
    ctx.close()
    best = [max(r["fitness"] for r in seg) for seg in res]
    home = [s for s, b in enumerate(boxes) if b[4] <= tau0_inj <= b[5]]
    assert home
    # the tile holding the injected chirp times reaches most of the injected SNR^2 = 144
    assert max(best[s] for s in home) > 0.8 * 144.0


def test_time_slide_background_returns_one_statistic_per_slide():
    import paper_2002_02150_gb300 as fc
    w = sd.SMALL
    data = sd.make_dataset(w, 35)
    t0lo, t0hi, t15lo, t15hi = sd.chirp_time_box(w.f_low)
    box = (0.0, 2 * math.pi, -0.5 * math.pi, 0.5 * math.pi, t0lo, t0hi, t15lo, t15hi)
    cfg = fc.pso_config(n_runs=2, n_particles=10, n_iter=20, seed=2, box=box)
    step = int(w.fs)                                        # 1 s
    shifts = np.array([[0, k * step, 2 * k * step, 3 * k * step] for k in range(4)])
    best, res = fc.time_slide_background(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low,
                                         w.f_high, shifts, cfg, max_batch=8)
    assert best.shape == (4,) and np.all(np.isfinite(best)) and np.all(best > 0)
    # slide k equals the search of a context made from the shifted data with segment k's seed
    k = 2
    ctx = fc.fcas_create(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high,
                         shifts=shifts[k])
    ref = fc.fcas_search(ctx, fc.pso_config(n_runs=2, n_particles=10, n_iter=20, seed=fc.segment_seed(2, k),
                                            box=box))
    ctx.close()
    assert res[k] == ref
