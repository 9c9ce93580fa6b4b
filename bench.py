"""Throughput of the batched coherent-fitness evaluation on one GB300 (or N, one rank per GPU).

One step = one fcas_fitness call over the whole batch of particles of the 4-detector x 60-min
@ 2048 Hz workload (7,372,800 samples zero-padded to 2^23, band 30-1000 Hz, 320 particles): sky
geometry, fused template x data x delay phase, both FFT passes over t_c, antenna projection and
argmax. ``value`` is particles evaluated per second over all ranks (weak scaling: every rank has
its own data realisation and particle batch, no data-path collective).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same workload.

Besides the contract keys the line carries: ``roofline`` (pass A's algorithmic bytes over its
CUDA-event time against the measured HBM copy rate, and its DRAM bytes from the committed ncu
record when that was taken on the current kernel sources), ``alu_view`` (algorithmic flops against
the FP32 issue peak), ``kernels`` (per-kernel times), ``fp64_form`` and ``ff_form`` (the binary64
and float-float forms on the same particles, with their differences from the FP32 form and from
each other), ``cufft_form`` (the straightforward cuFFT path), the PSO searches (``search``,
``paper_config_search``, ``search_60min`` and ``search_time_over_data_time``: the full 8 x 40 x 2000
search on the 60-min data, timed in full), ``differentiation`` (FP32 adjoint-gradient throughput and
gradient polishing), ``batched_uneven`` (64 segments of 15/30/60 min), the background and tiling
studies, and ``cpu_baseline`` (the oracle on the host cores, N = 1 only; the same leg evaluates the
oracle at the points the search and the polishing report).
"""

import argparse
import dataclasses
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthdata as sd  # noqa: E402

METRIC = "fitness evals/s (4 det x 60 min @2048 Hz, % HBM roofline); search time/data time"
UNIT = "evals/s"
PSO_EVALS = 8 * 40 * 2000          # 8 runs x 40 particles x 2000 iterations
DATA_SECONDS = 3600.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=sd.C2.name)
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="timed steps of the binary64 and float-float forms (0 = skip both)")
    ap.add_argument("--cpu-sample", type=int, default=1, help="particles per host core in the oracle CPU baseline")
    ap.add_argument("--particles", type=int, default=0, help="particles per GPU (0 = the workload's batch)")
    ap.add_argument("--max-batch", type=int, default=0, help="particles per internal chunk (0 = automatic)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end measurement")
    ap.add_argument("--paper-iters", type=int, default=500,
                    help="PSO iterations of the search in the paper's own configuration (0 = skip)")
    ap.add_argument("--background-slides", type=int, default=8,
                    help="time-shifted 64-s noise realisations of the background study (0 = skip)")
    ap.add_argument("--cufft-batches", type=int, default=2,
                    help="timed batches of 4 particles of the cuFFT comparison form (0 = skip)")
    ap.add_argument("--no-search", action="store_true", help="skip the PSO search measurements")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shape (no autotuning)")
    ap.add_argument("--group-segments", type=int, default=64,
                    help="segments of the batched uneven-length measurement (0 = skip)")
    ap.add_argument("--search-iters", type=int, default=2000,
                    help="PSO iterations of the timed 60-min search (the search-time ratio)")
    ap.add_argument("--no-gradient", action="store_true", help="skip the gradient and polishing measurements")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------- ranks
class Ranks:
    """Process-group plumbing: barrier and max/sum over ranks (gloo on CPU, nccl on GPUs)."""

    def __init__(self, backend=None):
        import torch
        import torch.distributed as dist
        self.dist = dist
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.on = self.world > 1 and backend != "none"
        if self.on and not dist.is_initialized():
            if backend is None:
                backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend=backend)
        self.backend = dist.get_backend() if self.on else None

    def _dev(self):
        import torch
        return torch.device("cuda", self.local) if self.backend == "nccl" else torch.device("cpu")

    def barrier(self):
        if self.on:
            self.dist.barrier()

    def reduce(self, value, op):
        if not self.on:
            return value
        import torch
        t = torch.tensor([float(value)], dtype=torch.float64, device=self._dev())
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX if op == "max" else self.dist.ReduceOp.SUM)
        return float(t.item())


def aggregate(ranks, local_units, local_seconds):
    """Whole-job throughput: units summed over ranks / slowest rank's time."""
    total = ranks.reduce(local_units, "sum")
    slowest = ranks.reduce(local_seconds, "max")
    return total / slowest, slowest


# ------------------------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------------------------------- roofline
FITNESS_KERNEL_SOURCES = ["paper_2002_02150_gb300/csrc/fcas_passes.cuh", "paper_2002_02150_gb300/csrc/fcas_kernels.cuh",
                          "paper_2002_02150_gb300/csrc/fcas_fft16.cuh", "paper_2002_02150_gb300/csrc/fcas_internal.cuh",
                          "paper_2002_02150_gb300/csrc/fcas_x2.cuh", "include/fcas.h"]


def _code_only(text):
    """C/C++ source without comments and with whitespace collapsed (edits to comments do not change
    the kernels)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash():
    """Hash of the code (comments excluded) the fitness kernels (pass A, pass B) are compiled from;
    of the public header only its macros (declarations of other entry points do not change them)."""
    h = hashlib.sha256()
    for p in FITNESS_KERNEL_SOURCES:
        text = _code_only(open(os.path.join(ROOT, p)).read())
        if p.endswith("fcas.h"):
            text = " ".join(ln for ln in open(os.path.join(ROOT, p)).read().splitlines() if ln.startswith("#define"))
        h.update(text.encode())
    return h.hexdigest()[:16]


# FP32 issue peak of the GB300 from the unit counts and the maximum SM clock: 152 SMs x 128 FP32
# lanes x 2 flops (fused multiply-add) x 2.07 GHz; binary64 at the nominal 1.25 TFLOP/s.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_NOMINAL_TFLOPS = 1.25


def flop_per_eval(n_fft, n_det, n_band):
    """Algorithmic flops of one evaluation: two complex transforms of length N (5 N log2 N each), the
    spectrum formation per band bin (per detector a complex product with the delay phasor and the
    two weighted accumulations, 14 flops; then the chirp phase, 8, and two complex products, 12),
    the inter-pass twiddle (one complex product per point of both series) and |W_1|^2 + |W_2|^2."""
    log_n = int(round(math.log2(n_fft)))
    return 2 * 5 * n_fft * log_n + n_band * (14 * n_det + 20) + 2 * 6 * n_fft + 4 * n_fft


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current kernels."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("kernel_hash") != kernel_source_hash():
        return None
    return e.get("bytes_per_launch")


# ------------------------------------------------------------------------------------------- workload
def workload_inputs(w, rank, particles=0):
    data = sd.make_dataset(w, seed=rank)
    theta = sd.make_particles(w, n=particles or None, seed=rank)
    return data, theta


def bench_ours(args, ranks):
    import torch
    import paper_2002_02150_gb300 as fc

    torch.cuda.set_device(ranks.local)
    dev = torch.device("cuda", ranks.local)
    w = sd.workload_by_name(args.workload)
    data, theta = workload_inputs(w, ranks.rank, args.particles)
    n = theta.shape[0]
    ctx = fc.fcas_create(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high, precision="fp32",
                         max_batch=args.max_batch)
    if not args.no_tune:
        fc.fcas_autotune(ctx, min(64, n))
    info = fc.fcas_get_info(ctx)
    th = torch.tensor(theta, device=dev)
    fit = torch.empty(n, dtype=torch.float64, device=dev)
    tc = torch.empty(n, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        fc.fcas_fitness(ctx, th, fit, tc, stream=stream.cuda_stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    fc.fcas_profile_enable(ctx, True)
    ranks.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(ranks.local)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    clock = clocks.stop()
    ranks.barrier()
    local_s = t0.elapsed_time(t1) / 1e3
    kern = {k: fc.fcas_profile_read(ctx, k) for k in ("geometry", "pass_a", "pass_b", "reduce")}
    fc.fcas_profile_enable(ctx, False)
    value, slowest = aggregate(ranks, n * args.steps, local_s)

    # roofline of the dominant kernel: algorithmic bytes per launch / mean launch time
    d, nn, nband = info["n_det"], info["n_fft"], info["n_band"]
    chunks_per_step = -(-n // info["chunk"])
    parts = [min(info["chunk"], n - c * info["chunk"]) for c in range(chunks_per_step)]
    mean_p = sum(parts) / len(parts)
    # pass A writes the two network-weighted series of every particle and reads the band spectrum
    # (D complex values per bin) and the chirp basis (one float-float pair per bin) once per
    # launch; pass B reads the series back
    algo = {"pass_a": mean_p * info["inter_bytes"] + (d + 1) * nband * 8, "pass_b": mean_p * info["inter_bytes"]}
    peak, peak_kind = measured_peak()
    dom = max(("pass_a", "pass_b"), key=lambda k: kern[k][0])
    ms, launches = kern[dom]
    achieved = algo[dom] / (ms / launches / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                "traffic": ncu_traffic(dom, w.name), "algorithmic_bytes_per_launch": int(algo[dom]),
                "launch_ms": round(ms / launches, 4)}
    kernels = {k: {"ms_total": round(v[0], 3), "launches": v[1]} for k, v in kern.items()}
    for k in ("pass_a", "pass_b"):
        if kern[k][1]:
            gbs = algo[k] / (kern[k][0] / kern[k][1] / 1e3) / 1e9
            kernels[k].update({"algorithmic_gbs": round(gbs, 1), "frac_of_measured_hbm": round(gbs / peak, 4)})
    gpu_launches = sum(v[1] for v in kern.values())

    # end to end through the C ABI with host buffers (pinned): H2D of theta, D2H of results
    e2e = None
    th_h = torch.tensor(theta).pin_memory()
    fit_h = torch.empty(n, dtype=torch.float64).pin_memory()
    tc_h = torch.empty(n, dtype=torch.int64).pin_memory()
    if not args.no_e2e:
        for _ in range(max(1, args.warmup)):
            fc.fcas_fitness(ctx, th_h, fit_h, tc_h, stream=stream.cuda_stream)
        ranks.barrier()
        torch.cuda.synchronize(dev)
        h0 = time.perf_counter()
        for _ in range(args.steps):
            fc.fcas_fitness(ctx, th_h, fit_h, tc_h, stream=stream.cuda_stream)
        torch.cuda.synchronize(dev)
        e2e_s = time.perf_counter() - h0
        ranks.barrier()
        e2e_value, _ = aggregate(ranks, n * args.steps, e2e_s)
        e2e = {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": int(th_h.numel() * 8),
               "d2h_bytes_per_step": int(n * 16)}
    ctx.close()

    cufft = None
    if args.cufft_batches > 0:
        ref = (fit.double().cpu().numpy(), tc.cpu().numpy())
        cufft = bench_cufft(w, data, theta, *ref, dev, steps=args.cufft_batches)
        cufft["fp64"] = bench_cufft(w, data, theta, *ref, dev, steps=args.cufft_batches, fp64=True)

    # plain binary64 form and the float-float form on the same workload (fewer steps: they are
    # binary64- and FP32-issue bound)
    fp64, ff = None, None
    if args.fp64_steps > 0:
        fit32, tc32 = fit.clone(), tc.clone()          # FP32-form results of the timed steps
        flop = flop_per_eval(w.n_fft, info["n_det"], info["n_band"])

        def time_form(precision):
            cx = fc.fcas_create(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high,
                                precision=precision, max_batch=args.max_batch)
            fc.fcas_fitness(cx, th, fit, tc, stream=stream.cuda_stream)
            ranks.barrier()
            torch.cuda.synchronize(dev)
            t0.record(stream)
            for _ in range(args.fp64_steps):
                fc.fcas_fitness(cx, th, fit, tc, stream=stream.cuda_stream)
            t1.record(stream)
            torch.cuda.synchronize(dev)
            cx.close()
            secs = t0.elapsed_time(t1) / 1e3
            v, _ = aggregate(ranks, n * args.fp64_steps, secs)
            return {"value": round(v, 2), "unit": UNIT, "steps": args.fp64_steps,
                    "ms_per_step": round(1e3 * secs / args.fp64_steps, 3)}, v, fit.clone(), tc.clone()

        def form_error(f_a, tc_a, f_ref, tc_ref):
            rel = ((f_a - f_ref).abs() / f_ref.abs()).double().cpu().numpy()
            return {"max_rel": float(rel.max()), "median_rel": float(np.median(rel)),
                    "same_tc_fraction": float((tc_a == tc_ref).double().mean().item()), "particles": n}

        fp64, v64, fit64, tc64 = time_form("fp64")
        tf64 = v64 * flop / 1e12
        fp64.update({"dtype": "f64",
                     "alu": {"bound": "alu", "achieved": round(tf64, 4), "peak": FP64_NOMINAL_TFLOPS,
                             "unit": "TFLOP/s", "frac": round(tf64 / FP64_NOMINAL_TFLOPS, 4),
                             "peak_source": "nominal binary64 rate"},
                     # error of the FP32 form (float-float phase) against the binary64 form
                     "fp32_form_error": form_error(fit32, tc32, fit64, tc64)})
        ff, _, fitff, tcff = time_form("ff")
        ff.update({"dtype": "f64 phase + float-float transforms",
                   "error_vs_fp64_form": form_error(fitff, tcff, fit64, tc64)})

    search = None if args.no_search else bench_search(fc, ranks, data, w, dev, args.search_iters)
    grad = None if (args.no_search or args.no_gradient) else bench_gradient(fc, ranks, dev,
                                                                              search["best_64s"]["snr10"])
    group = None if args.group_segments <= 0 else bench_group(fc, ranks, args.group_segments, dev)
    background, tiled = (None, None) if args.background_slides <= 0 else bench_background(fc, ranks, dev,
                                                                                        args.background_slides)
    paper_cfg = None if args.paper_iters <= 0 else bench_paper_config(fc, ranks, dev, args.paper_iters)

    out = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": ranks.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * slowest / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "detectors": list(w.detectors), "n_fft": w.n_fft, "n_samples": w.n_samples,
                   "fs": w.fs, "band_hz": [w.f_low, w.f_high], "particles_per_gpu": n,
                   "precision": "fp32 + float-float phase", "chunk": info["chunk"],
                   "shape": {"split_bias": info["split_bias"], "k1b": info["k1b"], "sub": info["sub"],
                             "autotuned": info["tuned_ms_per_particle"] > 0},
                   "l2": "inputs larger than L2 (intermediate %.1f GB per step), no flush" % (n * info["inter_bytes"] / 1e9)},
        "roofline": roofline,
        "alu_view": {"flop_per_eval": flop_per_eval(w.n_fft, d, nband),
                     "achieved": round(value / ranks.world * flop_per_eval(w.n_fft, d, nband) / 1e12, 3),
                     "peak": round(FP32_PEAK_TFLOPS, 2), "unit": "TFLOP/s",
                     "frac": round(value / ranks.world * flop_per_eval(w.n_fft, d, nband) / 1e12 / FP32_PEAK_TFLOPS, 4),
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                     "note": "whole fitness path per GPU; both passes issue-bound (see profiles/)"},
        "kernels": kernels, "gpu_launches": gpu_launches, "e2e": e2e, "clocks": clock,
        "fp64_form": fp64, "ff_form": ff, "cufft_form": cufft,
        "search_time_over_data_time": (search["search_time_over_data_time"] if search else
                                       {"value": round(PSO_EVALS / value / DATA_SECONDS, 5),
                                        "how": "extrapolated: 8 runs x 40 particles x 2000 iterations / value / 3600 s"}),
        "search": search["search_64s"] if search else None,
        "search_60min": search["search_60min"] if search else None,
        "differentiation": grad,
        "batched_uneven": group, "background_time_slides": background, "tiled_search": tiled,
        "paper_config_search": paper_cfg,
        "paper_context": {"search_over_data": [1.4, 0.5], "hardware": "1 KNL node per PSO run, FP64"},
    }
    if ranks.rank == 0 and ranks.world == 1 and args.cpu_sample > 0:      # the CPU baseline is an N = 1 figure
        judge = {}
        if search:
            judge["search_60min_best"] = (w.name, ranks.rank, {}, [search["search_60min"]["best_theta"]])
        if grad:
            pol = grad["polish"]
            d = pol["data"]
            judge["polish_before"] = (d["workload"], d["seed"], {"snr": d["snr"]}, pol["theta_before"])
            judge["polish_after"] = (d["workload"], d["seed"], {"snr": d["snr"]}, pol["theta_after"])
        out["cpu_baseline"] = cpu_baseline(w, ranks.rank, theta, args.cpu_sample, judge)
        jv = out["cpu_baseline"].get("judged_by_oracle", {})
        if "search_60min_best" in jv:
            out["search_60min"]["oracle_fitness_at_best"] = jv["search_60min_best"][0][0]
        if "polish_after" in jv:
            before = np.array([v for v, _ in jv["polish_before"]])
            after = np.array([v for v, _ in jv["polish_after"]])
            out["differentiation"]["polish"]["oracle_gain"] = {
                "fitness_before": [round(float(v), 4) for v in before],
                "fitness_after": [round(float(v), 4) for v in after],
                "gain": [round(float(v), 5) for v in after - before],
                "mean_relative_gain": float(np.mean((after - before) / before)),
                "how": "FP64 oracle fitness at each run's best particle before and after 10 fcas_polish steps"}
    if grad:
        for k in ("theta_before", "theta_after", "data"):
            grad["polish"].pop(k, None)
    return out


C_LIGHT = 299792458.0


def _chirp_coefficients(tau0, tau15, f_star):
    """Chirp-phase coefficients in turns for the powers phi^-5/3, phi^-1, phi^-2/3, phi^-1/3 of
    phi = f / f_* (restricted 2PN phase in chirp times, Sec. II.B)."""
    x = 5.0 * tau15 / (32.0 * np.pi * tau0)
    eta = x ** (-2.0 / 3.0) / (8.0 * f_star * tau15)
    tau1 = 5.0 / (192.0 * np.pi * f_star * eta * x) * (743.0 / 336.0 + 11.0 * eta / 4.0)
    tau2 = 5.0 / (128.0 * np.pi * f_star * eta * x ** (1.0 / 3.0)) * (
        3058673.0 / 1016064.0 + 5429.0 * eta / 1008.0 + 617.0 * eta ** 2 / 144.0)
    return 0.6 * f_star * tau0, f_star * tau1, -1.5 * f_star * tau15, 3.0 * f_star * tau2


def bench_cufft(w, data, theta, fit_ref, tc_ref, dev, batch=4, steps=2, fp64=False):
    """The straightforward GPU form, timed for comparison: per particle and detector the spectrum
    Q_i[k] = 4 df y~^i[k] e^{2 pi i f_k Delta^i} h~_c*[k] is formed by PyTorch element-wise kernels
    (binary64 phase, complex64 product; complex128 throughout with fp64), transformed by cuFFT
    (torch.fft.ifft, complex64 or complex128, length N,
    one transform per detector), then projected, Gamma^2(t) = X_c^T G^-1 X_c + X_s^T G^-1 X_s, and
    maximised over t, each a separate kernel (the projection through the Cholesky factor of G^-1,
    as a sum of squares). Its results are compared with the fused path's."""
    import torch
    cdt, rdt = (torch.complex128, torch.float64) if fp64 else (torch.complex64, torch.float32)
    d9 = np.asarray(data["det"], dtype=np.float64)
    n_det, n, fs = d9.shape[0], w.n_fft, w.fs
    df = fs / n
    kk = torch.arange(n // 2 + 1, device=dev)
    f_all = kk.double() * df
    kf = kk.double() * fs                                    # band f_low < f <= f_high, 0 < k < N/2
    sel = ((kf > w.f_low * n) & (kf <= w.f_high * n) & (kk > 0) & (kk < n // 2)).nonzero().squeeze(1)
    f = f_all[sel]
    x = torch.zeros(n_det, n, dtype=torch.float64, device=dev)
    x[:, : w.n_samples] = torch.as_tensor(np.asarray(data["data"]), device=dev)
    psd = torch.as_tensor(np.asarray(data["psd"]), device=dev)[:, sel]
    y = torch.fft.rfft(x, dim=1)[:, sel] / fs / psd
    del x
    sigma2 = (4.0 * df * (f ** (-7.0 / 3.0))[None, :] / psd).sum(1).cpu().numpy()
    ybase = y * (4.0 * df * f ** (-7.0 / 6.0))[None, :] * np.exp(-0.25j * np.pi)
    del y, psd
    phi = f / w.f_low
    powers = torch.stack([phi ** (-5.0 / 3.0), 1.0 / phi, phi ** (-2.0 / 3.0), phi ** (-1.0 / 3.0)])

    def geometry(th):
        a, dlt = th[0], th[1]
        sa, ca, sd_, cd = np.sin(a), np.cos(a), np.sin(dlt), np.cos(dlt)
        nhat = np.array([cd * ca, cd * sa, sd_])
        bx, by = np.array([sa, -ca, 0.0]), np.array([-sd_ * ca, -sd_ * sa, cd])
        xX, xY, yX, yY = d9[:, 3:6] @ bx, d9[:, 3:6] @ by, d9[:, 6:9] @ bx, d9[:, 6:9] @ by
        u = np.stack([0.5 * (xX * xX - xY * xY - yX * yX + yY * yY), xX * xY - yX * yY], axis=1)
        g = (u * sigma2[:, None]).T @ u
        det = g[0, 0] * g[1, 1] - g[0, 1] ** 2
        tr = g[0, 0] + g[1, 1]
        if det < 1e-12 * (0.5 * tr) ** 2:
            ev, vec = np.linalg.eigh(g)
            chol = np.stack([vec[:, 1] / np.sqrt(ev[1]), np.zeros(2)], axis=1)      # G^-1 = e e^T / lambda
        else:
            chol = np.linalg.cholesky(np.array([[g[1, 1], -g[0, 1]], [-g[0, 1], g[0, 0]]]) / det)
        # Gamma^2 = |L^T X_c|^2 + |L^T X_s|^2 with L L^T = G^-1: the detector weights u L
        return -(d9[:, 0:3] @ nhat) / C_LIGHT, u @ chol

    def run(ths):
        b = len(ths)
        geo = [geometry(th) for th in ths]
        coef = torch.tensor([_chirp_coefficients(th[2], th[3], w.f_low) for th in ths], device=dev)
        delay = torch.tensor(np.stack([g[0] for g in geo]), device=dev)
        wts = torch.tensor(np.stack([g[1] for g in geo]), device=dev, dtype=rdt)
        turns = (coef @ powers)[:, None, :] + delay[:, :, None] * f[None, None, :]
        turns = turns - torch.round(turns)
        q = (ybase[None] * torch.polar(torch.ones_like(turns), 2.0 * np.pi * turns)).to(cdt)
        full = torch.zeros(b, n_det, n, dtype=cdt, device=dev)
        full[:, :, sel] = q
        del q, turns
        z = torch.fft.ifft(full, dim=-1) * n
        del full
        xc = torch.einsum("bia,bit->bat", wts, z.real)
        xs = torch.einsum("bia,bit->bat", wts, z.imag)
        del z
        g2 = (xc * xc + xs * xs).sum(1)
        val, idx = g2[:, : w.n_samples].max(dim=1)
        return val, idx

    m = batch * steps
    ths = [theta[j % len(theta)] for j in range(m)]
    run(ths[:batch])                          # cuFFT plan and allocator warm-up
    gpu = dev.type == "cuda"
    if gpu:
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
    h0 = time.perf_counter()
    outs = [run(ths[batch * s: batch * (s + 1)]) for s in range(steps)]
    if gpu:
        e1.record()
        torch.cuda.synchronize(dev)
        sec = e0.elapsed_time(e1) / 1e3
    else:
        sec = time.perf_counter() - h0
    vals = torch.cat([o[0] for o in outs]).double().cpu().numpy()
    idx = torch.cat([o[1] for o in outs]).cpu().numpy()
    ref = np.asarray(fit_ref)[[j % len(theta) for j in range(m)]]
    rel = float(np.max(np.abs(vals - ref) / np.abs(ref)))
    same_tc = float(np.mean(idx == np.asarray(tc_ref)[[j % len(theta) for j in range(m)]]))
    return {"value": round(m / sec, 2), "unit": UNIT, "particles": m,
            "max_rel_diff_vs_fused": rel, "same_tc_fraction": same_tc,
            "how": "torch element-wise kernels (binary64 phase) + cuFFT %s inverse transforms of length N "
                   "per detector + einsum projection + max, %d particles per batch"
                   % ("complex128" if fp64 else "complex64", batch)}


def _pso_box(w):
    t0lo, t0hi, t15lo, t15hi = sd.chirp_time_box(w.f_low)
    return (0.0, 2 * 3.141592653589793, -0.5 * 3.141592653589793, 0.5 * 3.141592653589793, t0lo, t0hi, t15lo, t15hi)


def bench_search(fc, ranks, data60, w60, dev, iters60=2000):
    """Full PSO searches: 8 lbest-ring runs x 40 particles x 2000 iterations on the 64-s data (an SNR-10
    and an SNR-12 injection and a noise-only realisation), and the same search on the 60-min data of
    the fitness benchmark (SNR-10 injection), timed in full: its wall time over the 3600-s data
    duration is the search-time ratio."""
    import torch
    w = sd.C1
    runs = []
    best_64s = {}
    for kind, kw in (("snr10", dict(snr=10.0)), ("snr12", dict(snr=12.0)), ("noise", dict(inject=False))):
        data = sd.make_dataset(w, seed=10 + ranks.rank, **kw)
        ctx = fc.fcas_create(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high)
        cfg = fc.pso_config(n_runs=8, n_particles=40, n_iter=2000, seed=2020 + ranks.rank, box=_pso_box(w))
        fc.fcas_search(ctx, fc.pso_config(n_runs=8, n_particles=40, n_iter=3, seed=1, box=_pso_box(w)))  # warm-up
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        res = fc.fcas_search(ctx, cfg)
        wall = time.perf_counter() - t
        best = max(res, key=lambda r: r["fitness"])
        best_64s[kind] = res
        entry = {"realisation": kind, "wall_s": round(wall, 3), "wall_over_data": round(wall / (w.n_samples / w.fs), 4),
                 "evaluations": int(sum(r["evaluations"] for r in res)), "best_fitness": best["fitness"],
                 "best_theta": [round(v, 6) for v in best["theta"]], "best_tc_s": best["tc"] / w.fs}
        if data["inj"] is not None:
            entry["injected"] = _injected(fc, ctx, w, data["inj"])
        ctx.close()
        runs.append(entry)
    # the 60-min segment, all iterations timed
    ctx = fc.fcas_create(data60["det"], data60["psd"], data60["data"], w60.n_fft, w60.fs, w60.f_low, w60.f_high)
    fc.fcas_autotune(ctx, 64)
    fc.fcas_search(ctx, fc.pso_config(n_runs=8, n_particles=40, n_iter=3, seed=1, box=_pso_box(w60)))   # warm-up
    torch.cuda.synchronize(dev)
    t = time.perf_counter()
    res = fc.fcas_search(ctx, fc.pso_config(n_runs=8, n_particles=40, n_iter=iters60, seed=3 + ranks.rank,
                                            box=_pso_box(w60)))
    wall = time.perf_counter() - t
    best = max(res, key=lambda r: r["fitness"])
    search60 = {"workload": w60.name, "runs": 8, "particles": 40, "iterations": iters60, "wall_s": round(wall, 3),
                "evaluations": int(sum(r["evaluations"] for r in res)),
                "evals_per_s": round(sum(r["evaluations"] for r in res) / wall, 1),
                "best_fitness": best["fitness"], "best_theta": [round(v, 6) for v in best["theta"]],
                "best_tc_s": best["tc"] / w60.fs, "run_best_fitness": [round(r["fitness"], 3) for r in res],
                "injected": _injected(fc, ctx, w60, data60["inj"]) if data60["inj"] is not None else None}
    ctx.close()
    ratio = {"value": round(wall / DATA_SECONDS, 5),
             "how": f"60-min data, 8 runs x 40 particles x {iters60} iterations, measured in full ({wall:.2f} s) "
                    "/ 3600 s"}
    return {"search_64s": {"workload": w.name, "runs": 8, "particles": 40, "iterations": 2000, "realisations": runs},
            "search_60min": search60, "search_time_over_data_time": ratio, "best_64s": best_64s}


def bench_gradient(fc, ranks, dev, best_runs, steps=5):
    """Differentiation form (64-s data): the adjoint gradient of 320 particles in the FP32 form, timed
    on the device, and 10 steps of gradient polishing (fcas_polish) of each PSO run's best particle of
    the SNR-10 search. The polished points are judged by the FP64 oracle in the CPU-baseline leg."""
    import torch
    w = sd.C1
    data = sd.make_dataset(w, seed=10 + ranks.rank, snr=10.0)
    ctx = fc.fcas_create(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high)
    th = torch.tensor(sd.make_particles(w, 320, seed=1), device=dev)
    fit, tc = fc.fcas_fitness(ctx, th)
    grad = torch.empty((320, 4), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        fc.fcas_gradient(ctx, th, tc, grad, stream=stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fc.fcas_gradient(ctx, th, tc, grad, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    sec = e0.elapsed_time(e1) / 1e3
    start = np.array([r["theta"] for r in best_runs])
    f0, _ = fc.fcas_fitness(ctx, start)
    torch.cuda.synchronize(dev)
    t = time.perf_counter()
    th_p, f_p, tc_p, acc = fc.fcas_polish(ctx, start, steps=10)
    polish_s = time.perf_counter() - t
    ctx.close()
    return {"gradient": {"workload": w.name, "particles": 320, "precision": "fp32",
                         "value": round(320 * steps / sec, 1), "unit": "gradients/s",
                         "ms_per_call": round(1e3 * sec / steps, 3)},
            "polish": {"workload": w.name, "points": len(start), "steps": 10, "wall_s": round(polish_s, 4),
                       "fitness_before": [round(float(v), 4) for v in f0],
                       "fitness_after": [round(float(v), 4) for v in f_p], "accepted_steps": [int(a) for a in acc],
                       "theta_before": start.tolist(), "theta_after": th_p.tolist(),
                       "data": {"workload": w.name, "seed": 10 + ranks.rank, "snr": 10.0}}}


def bench_background(fc, ranks, dev, n_slides):
    """Small-scale H0 study (Sec. V background by time shifts) and chirp-time tiling (Sec. IV): the
    full search (8 runs x 40 particles x 2000 iterations) on n_slides time-shifted copies of one
    noise-only 64-s realisation (detector i of slide k shifted by 10 k i s, circularly), all slides
    in one group; and the SNR-10 injection searched over a 2 x 2 tiling of the chirp-time box."""
    import torch
    w = sd.C1
    box = _pso_box(w)
    cfg = fc.pso_config(n_runs=8, n_particles=40, n_iter=2000, seed=4040 + ranks.rank, box=box)
    data = sd.make_dataset(w, seed=40 + ranks.rank, inject=False)
    step = int(round(10.0 * w.fs))
    shifts = np.array([[k * i * step for i in range(w.n_det)] for k in range(1, n_slides + 1)])
    torch.cuda.synchronize(dev)
    t = time.perf_counter()
    best, res = fc.time_slide_background(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high,
                                         shifts, cfg)
    wall = time.perf_counter() - t
    evals = int(sum(r["evaluations"] for seg in res for r in seg))
    q = np.sort(best)
    background = {"workload": w.name, "slides": n_slides, "shift_step_s": 10.0, "evaluations": evals,
                  "wall_s": round(wall, 3), "evals_per_s": round(evals / wall, 1),
                  "max_statistic_per_slide": [round(float(v), 3) for v in best],
                  "median": round(float(np.median(q)), 3),
                  "threshold_fap_1_over_slides": round(float(q[-1]), 3),
                  "how": "best Gamma^2 over 8 runs per slide; the largest of the slides is the empirical threshold "
                         "at a false-alarm probability of 1/slides per 64-s segment"}
    # chirp-time tiling of the SNR-10 injection
    d10 = sd.make_dataset(w, seed=10 + ranks.rank, snr=10.0)
    boxes = fc.fcas_tau_tiles(box[4], box[5], box[6], box[7], 2, 2, 0.1)
    ctx = fc.fcas_create(d10["det"], d10["psd"], d10["data"], w.n_fft, w.fs, w.f_low, w.f_high,
                         flags=fc.FCAS_SETUP_LAZY_SCRATCH)
    with fc.fcas_group_create([ctx] * len(boxes)) as grp:
        grp.search(fc.pso_config(n_runs=8, n_particles=40, n_iter=3, seed=1, box=box), boxes=boxes)   # warm-up
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        tres = grp.search(cfg, boxes=boxes)
        twall = time.perf_counter() - t
    ctx.close()
    tiled = {"workload": w.name, "tiles": "2 x 2, overlap 0.1", "wall_s": round(twall, 3),
             "best_per_tile": [round(max(r["fitness"] for r in seg), 3) for seg in tres],
             "boxes_tau": [[round(b[4], 4), round(b[5], 4), round(b[6], 5), round(b[7], 5)] for b in boxes],
             "injected_snr2": 100.0}
    return background, tiled


def bench_paper_config(fc, ranks, dev, n_iter):
    """The paper's own search configuration (Sec. V): 60 min of 4-detector data at 2048 Hz with
    f_* = 10 Hz, a 1.5 + 1.5 Msun signal arriving 20 min into the data at network SNR 12, searched
    with the paper's tuned settings for SNR >= 12 (12 lbest runs x 40 particles, 500 iterations) over
    the whole sky and tau0 in [500, 1500] s, tau1.5 in [5, 15] s."""
    import torch
    w = sd.PAPER_DNS
    data = sd.make_dataset(w, seed=80 + ranks.rank)
    box = (0.0, 2 * math.pi, -0.5 * math.pi, 0.5 * math.pi) + tuple(sd.PAPER_TAU_BOX)
    ctx = fc.fcas_create(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high)
    fc.fcas_autotune(ctx, 64)
    fc.fcas_search(ctx, fc.pso_config(n_runs=12, n_particles=40, n_iter=3, seed=1, box=box))   # warm-up
    torch.cuda.synchronize(dev)
    t = time.perf_counter()
    res = fc.fcas_search(ctx, fc.pso_config(n_runs=12, n_particles=40, n_iter=n_iter, seed=1010 + ranks.rank,
                                            box=box))
    wall = time.perf_counter() - t
    best = max(res, key=lambda r: r["fitness"])
    out = {"workload": w.name, "f_star_hz": w.f_low, "tau_box": list(sd.PAPER_TAU_BOX), "runs": 12, "particles": 40,
           "iterations": n_iter, "wall_s": round(wall, 3), "wall_over_data": round(wall / (w.n_samples / w.fs), 5),
           "evaluations": int(sum(r["evaluations"] for r in res)), "best_fitness": best["fitness"],
           "best_theta": [round(v, 6) for v in best["theta"]], "best_tc_s": best["tc"] / w.fs,
           "run_best_fitness": [round(r["fitness"], 3) for r in res],
           "injected": _injected(fc, ctx, w, data["inj"])}
    ctx.close()
    return out


def _injected(fc, ctx, w, inj):
    """The injected parameters (chirp times from the injected masses) and the library's fitness there."""
    t0, t15 = sd.workloads._chirp_times_tau0_tau15(inj["m1"], inj["m2"], w.f_low)
    f, t = fc.fcas_fitness(ctx, np.array([[inj["alpha"], inj["delta"], t0, t15]]))
    return {"alpha": round(inj["alpha"], 6), "delta": round(inj["delta"], 6), "tau0": round(t0, 6),
            "tau15": round(t15, 6), "tc_s": inj["t_c"], "snr2": inj["snr"] ** 2,
            "fitness_at_injection": float(f[0]), "tc_s_at_injection": float(t[0]) / w.fs}


def _segment_workload(seg, rng_draws):
    """Segment seg of the uneven-length batch: durations cycled over 15/30/60 min at 2048 Hz (FFT
    lengths 2^21, 2^22, 2^23), masses and SNR from the given draws (m1, m2, snr)."""
    minutes, n_fft = ((15, 1 << 21), (30, 1 << 22), (60, 1 << 23))[seg % 3]
    n_samples = minutes * 60 * 2048
    m1, m2, snr = rng_draws
    return dataclasses.replace(sd.C2, name=f"{minutes}min", n_samples=n_samples, n_fft=n_fft, m1=float(m1),
                               m2=float(m2), snr=float(snr), arrival_s=n_samples / 2048.0 / 3.0)


def _segment_data(args):
    """Worker of the segment data pool: the seeded data of one segment (data and detector table)."""
    seg, draws, seed = args
    d = sd.make_dataset(_segment_workload(seg, draws), seed=seed)
    return seg, d["data"], d["det"]


def bench_group(fc, ranks, n_seg, dev, iters=5):
    """Uneven batching: n_seg noise realisations with DNS injections (SNR ~ U[10, 14], masses ~ U[1, 3]
    Msun, random sky), durations cycled over 15/30/60 min at 2048 Hz (FFT lengths 2^21, 2^22, 2^23),
    every segment's swarm (8 runs x 40 particles) advanced together, one graph launch per iteration,
    each segment with autotuned launch shapes and the library's analytic PSD (psd = NULL). The seeded
    data of the segments is generated by a pool of spawned host processes."""
    import multiprocessing as mp
    import tempfile
    import torch
    rng = np.random.default_rng(4000 + ranks.rank)
    draws = [(*rng.uniform(1.0, 3.0, 2), rng.uniform(10.0, 14.0)) for _ in range(n_seg)]
    cache = os.path.join(tempfile.gettempdir(), f"fcas_tune_rank{ranks.rank}.txt")
    ctxs, lengths = [None] * n_seg, [0] * n_seg
    workers = max(1, min(n_seg, os.cpu_count() or 1, 16))
    avail = _mem_available_bytes()
    if avail:
        workers = max(1, min(workers, int(avail * 0.4 // 2.5e9)))
    t_data = time.perf_counter()
    jobs = [(s_, draws[s_], 500 + 64 * ranks.rank + s_) for s_ in range(n_seg)]
    with mp.get_context("spawn").Pool(workers) as pool:
        for s_, data, det in pool.imap_unordered(_segment_data, jobs):
            w = _segment_workload(s_, draws[s_])
            ctx = fc.fcas_create(det, None, data, w.n_fft, w.fs, w.f_low, w.f_high, flags=fc.FCAS_SETUP_LAZY_SCRATCH)
            fc.fcas_autotune(ctx, 64, cache)
            ctxs[s_], lengths[s_] = ctx, w.n_fft
            del data
    prep_s = time.perf_counter() - t_data
    cfg = lambda it: fc.pso_config(n_runs=8, n_particles=40, n_iter=it, seed=7, box=_pso_box(sd.C2))
    with fc.fcas_group_create(ctxs) as grp:
        grp.search(cfg(2))                      # warm-up (also builds the iteration graph once)
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        res = grp.search(cfg(iters))
        wall = time.perf_counter() - t
    shapes = [fc.fcas_get_info(c) for c in ctxs]
    for c in ctxs:
        c.close()
    evals = sum(r["evaluations"] for seg in res for r in seg)
    return {"segments": n_seg, "fft_lengths": lengths, "runs_per_segment": 8, "particles": 40, "iterations": iters,
            "evaluations_per_iteration": int(evals // iters), "wall_s": round(wall, 4),
            "s_per_iteration": round(wall / iters, 5), "evals_per_s": round(evals / wall, 1),
            "evaluations": int(evals), "data_and_contexts_s": round(prep_s, 2), "data_workers": workers,
            "psd": "analytic aLIGO fit evaluated by the library (psd = NULL)",
            "shapes": [{k: i[k] for k in ("n_fft", "split_bias", "k1b", "sub")} for i in shapes[:3]]}


def _oracle_worker(wname, seed, thetas, barrier, queue):
    """One host core of the oracle baseline: the oracle's own data preparation, then one particle
    per step, every step starting on all workers together."""
    try:
        from oracle import fcas_oracle as o
        w = sd.workload_by_name(wname)
        data = sd.make_dataset(w, seed=seed)
        setup = o.OracleSetup(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high)
        times = []
        for th in thetas:
            barrier.wait(timeout=900)
            t = time.perf_counter()
            o.fitness(setup, th)
            times.append(time.perf_counter() - t)
        queue.put(("ok", times))
    except Exception as e:  # reported to the parent, which then stops the pool
        queue.put(("error", repr(e)))


def _mem_available_bytes():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return None


ORACLE_WORKER_BYTES = 3.0e9     # peak resident size of one oracle worker on the 60-min workload


def oracle_pool(w, seed, theta, steps):
    """Times the FP64 oracle on the host cores: one spawned single-threaded process per core (as
    many as memory allows), each evaluating one particle per step. Returns (evals/s over all
    steps, workers, seconds per step); a step lasts as long as its slowest worker."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    avail = _mem_available_bytes()
    if avail:
        n = min(n, max(1, int(avail * 0.6 // (ORACLE_WORKER_BYTES if w.n_fft >= 1 << 22 else 0.5e9))))
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(n)
    queue = ctx.Queue()
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    procs = [ctx.Process(target=_oracle_worker,
                         args=(w.name, seed, [theta[(i + k * n) % len(theta)] for k in range(steps)], barrier, queue))
             for i in range(n)]
    try:
        for p in procs:
            p.start()
        results = []
        for _ in procs:
            status, val = queue.get(timeout=1800)
            if status != "ok":
                raise RuntimeError("oracle worker failed: " + val)
            results.append(val)
    finally:
        for p in procs:
            p.join(timeout=5)
            if p.is_alive():
                p.terminate()
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    step_s = [max(r[k] for r in results) for k in range(steps)]
    return n, step_s


def oracle_judgements(judge):
    """Part of the CPU-baseline leg: the FP64 oracle's fitness (and argmax) at points the GPU legs
    report, each on its own seeded workload. judge: {name: (workload name, seed, make_dataset
    keywords, [theta, ...])}."""
    from oracle import fcas_oracle as o
    out = {}
    setups = {}
    for name, (wname, seed, kw, thetas) in judge.items():
        key = (wname, seed, tuple(sorted(kw.items())))
        if key not in setups:
            w = sd.workload_by_name(wname)
            data = sd.make_dataset(w, seed=seed, **kw)
            setups[key] = o.OracleSetup(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high)
        out[name] = [list(o.fitness(setups[key], np.asarray(th, dtype=np.float64))) for th in thetas]
    return out


def cpu_baseline(w, seed, theta, steps, judge=None):
    n, step_s = oracle_pool(w, seed, theta, steps)
    value = n * steps / sum(step_s)
    out = {"value": round(value, 4), "unit": UNIT, "cores": n, "kind": "oracle",
           "sample": f"{n * steps} particles of the same workload ({steps} per core), FP64 numpy oracle, "
                     f"{n} single-threaded processes, data preparation excluded",
           "s_per_eval_per_core": round(n / value, 3),
           "search_s_extrapolated": {"value": round(PSO_EVALS / value, 1),
                                     "how": "8 runs x 40 particles x 2000 iterations / value (extrapolated, not run)"}}
    if judge:
        t = time.perf_counter()
        out["judged_by_oracle"] = oracle_judgements(judge)
        out["judge_s"] = round(time.perf_counter() - t, 2)
    return out


def bench_reference(args, ranks):
    w = sd.workload_by_name(args.workload)
    if ranks.rank != 0:          # under torchrun only rank 0 times the oracle; the others do no work
        return None
    theta = sd.make_particles(w, seed=0)
    n, step_s = oracle_pool(w, 0, theta, args.warmup + args.steps)
    timed = step_s[args.warmup:]
    value = n * args.steps / sum(timed)
    return {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ranks.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sum(timed) / args.steps, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n_fft": w.n_fft, "n_samples": w.n_samples,
                       "particles_per_step": n},
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": n, "kind": "oracle",
                             "sample": f"{n} particles of the workload per step (one per core), FP64 numpy oracle, "
                                       "single-threaded processes, data preparation excluded"},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.impl == "reference":
        ranks = Ranks(backend="none")
        out = bench_reference(args, ranks)
    else:
        ranks = Ranks()
        out = bench_ours(args, ranks)
    if ranks.rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if ranks.on:
        ranks.dist.destroy_process_group()


if __name__ == "__main__":
    main()
