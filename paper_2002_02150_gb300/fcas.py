"""Python binding of libfcas (argument marshalling only; every computation runs in the library).

Functions carry the C names: ``fcas_create``, ``fcas_fitness``, ``fcas_gradient``, ``fcas_polish``,
``fcas_search``, ``fcas_destroy``, ``fcas_last_error``, ``fcas_get_info``, ``fcas_profile_enable``,
``fcas_profile_read`` and the others of include/fcas.h.
Arrays may be numpy arrays (host memory) or torch CUDA tensors (device memory); device arrays make
the call asynchronous on the given stream (default: torch's current stream).
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FCAS_LIBRARY selects another build of the same library (the index-checked build of the tests)
LIB_PATH = os.environ.get("FCAS_LIBRARY") or os.path.join(_HERE, "libfcas.so")

FCAS_MAX_DET = 8
FCAS_PREC_FP64 = 0
FCAS_PREC_FP32 = 1
FCAS_PREC_FF = 2      # float-float transforms: binary64-class accuracy on the FP32 units
KERNEL_KINDS = {"geometry": 0, "pass_a": 1, "pass_b": 2, "reduce": 3}


class FcasError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libfcas error {code}: {msg}")
        self.code = code


class fcas_detector(ctypes.Structure):
    _fields_ = [("r", ctypes.c_double * 3), ("xarm", ctypes.c_double * 3), ("yarm", ctypes.c_double * 3)]


class fcas_setup(ctypes.Structure):
    _fields_ = [("n_det", ctypes.c_int32), ("precision", ctypes.c_int32), ("n_samples", ctypes.c_int64),
                ("n_fft", ctypes.c_int64), ("fs", ctypes.c_double), ("f_low", ctypes.c_double),
                ("f_high", ctypes.c_double), ("max_batch", ctypes.c_int32), ("flags", ctypes.c_int32)]


class fcas_info(ctypes.Structure):
    _fields_ = [("n_fft", ctypes.c_int64), ("n1", ctypes.c_int64), ("n2", ctypes.c_int64),
                ("k_lo", ctypes.c_int64), ("k_hi", ctypes.c_int64), ("n_band", ctypes.c_int64),
                ("chunk", ctypes.c_int64), ("n_det", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("scale", ctypes.c_double), ("sigma2", ctypes.c_double * FCAS_MAX_DET),
                ("inter_bytes", ctypes.c_int64), ("series", ctypes.c_int64), ("split_bias", ctypes.c_int32),
                ("k1b", ctypes.c_int32), ("sub", ctypes.c_int32), ("radix_bits_a", ctypes.c_int32),
                ("tuned_ms_per_particle", ctypes.c_double)]


class fcas_pso_config(ctypes.Structure):
    _fields_ = [("n_runs", ctypes.c_int32), ("n_particles", ctypes.c_int32), ("n_iter", ctypes.c_int32),
                ("n_neighbours", ctypes.c_int32), ("seed", ctypes.c_uint64), ("box", ctypes.c_double * 8),
                ("w_start", ctypes.c_double), ("w_end", ctypes.c_double), ("c1", ctypes.c_double),
                ("c2", ctypes.c_double), ("vmax", ctypes.c_double)]


class fcas_pso_state(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("v", ctypes.c_void_p), ("pbest_x", ctypes.c_void_p),
                ("pbest_f", ctypes.c_void_p), ("pbest_tc", ctypes.c_void_p)]


class fcas_search_result(ctypes.Structure):
    _fields_ = [("fitness", ctypes.c_double), ("theta", ctypes.c_double * 4), ("tc", ctypes.c_int64),
                ("evaluations", ctypes.c_int64)]


_lib = None


def load_library():
    """Load libfcas.so; raise if it has not been built (there is no fallback implementation)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.fcas_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(fcas_setup), ctypes.POINTER(fcas_detector),
                                vp, vp, vp]
    lib.fcas_create.restype = i32
    lib.fcas_fitness.argtypes = [vp, i64, vp, vp, vp, vp]
    lib.fcas_fitness.restype = i32
    lib.fcas_fitness_noalloc.argtypes = [vp, i64, vp, vp, vp, vp]
    lib.fcas_fitness_noalloc.restype = i32
    lib.fcas_destroy.argtypes = [vp]
    lib.fcas_destroy.restype = None
    lib.fcas_last_error.argtypes = []
    lib.fcas_last_error.restype = ctypes.c_char_p
    lib.fcas_version.argtypes = []
    lib.fcas_version.restype = i32
    lib.fcas_get_info.argtypes = [vp, ctypes.POINTER(fcas_info)]
    lib.fcas_get_info.restype = i32
    lib.fcas_profile_enable.argtypes = [vp, i32]
    lib.fcas_profile_enable.restype = i32
    lib.fcas_profile_read.argtypes = [vp, i32, ctypes.POINTER(dp), ctypes.POINTER(i64)]
    lib.fcas_profile_read.restype = i32
    lib.fcas_pso_init.argtypes = [ctypes.POINTER(fcas_pso_config), ctypes.POINTER(fcas_pso_state), vp]
    lib.fcas_pso_init.restype = i32
    lib.fcas_pso_update.argtypes = [ctypes.POINTER(fcas_pso_config), ctypes.c_int32, vp, vp,
                                    ctypes.POINTER(fcas_pso_state), vp]
    lib.fcas_pso_update.restype = i32
    lib.fcas_pso_theta.argtypes = [ctypes.POINTER(fcas_pso_config), vp, vp, vp]
    lib.fcas_pso_theta.restype = i32
    lib.fcas_search.argtypes = [vp, ctypes.POINTER(fcas_pso_config), ctypes.POINTER(fcas_search_result), vp]
    lib.fcas_search.restype = i32
    lib.fcas_gradient.argtypes = [vp, i64, vp, vp, vp, vp]
    lib.fcas_gradient.restype = i32
    lib.fcas_autotune.argtypes = [vp, i64, ctypes.c_char_p, vp]
    lib.fcas_autotune.restype = i32
    lib.fcas_set_shape.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp]
    lib.fcas_set_shape.restype = i32
    lib.fcas_group_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int32, ctypes.POINTER(vp), ctypes.c_int32]
    lib.fcas_group_create.restype = i32
    lib.fcas_group_search.argtypes = [vp, ctypes.POINTER(fcas_pso_config), ctypes.POINTER(fcas_search_result), vp]
    lib.fcas_group_search.restype = i32
    lib.fcas_group_destroy.argtypes = [vp]
    lib.fcas_group_destroy.restype = None
    lib.fcas_create_time_shifted.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(fcas_setup),
                                             ctypes.POINTER(fcas_detector), vp, vp, ctypes.POINTER(i64), vp]
    lib.fcas_create_time_shifted.restype = i32
    lib.fcas_group_search_boxes.argtypes = [vp, ctypes.POINTER(fcas_pso_config), ctypes.POINTER(dp),
                                            ctypes.POINTER(fcas_search_result), vp]
    lib.fcas_group_search_boxes.restype = i32
    lib.fcas_tau_tiles.argtypes = [dp, dp, dp, dp, ctypes.c_int32, ctypes.c_int32, dp, ctypes.POINTER(dp)]
    lib.fcas_tau_tiles.restype = i32
    lib.fcas_condition_number.argtypes = [vp, i64, vp, vp, vp]
    lib.fcas_condition_number.restype = i32
    lib.fcas_polish.argtypes = [vp, i64, vp, vp, vp, ctypes.c_int32, ctypes.POINTER(dp), ctypes.c_int32, vp, vp]
    lib.fcas_polish.restype = i32
    _lib = lib
    return lib


def fcas_last_error():
    return load_library().fcas_last_error().decode()


def _check(rc):
    if rc != 0:
        raise FcasError(rc, fcas_last_error())


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """Pointer to a contiguous array of the given numpy dtype (host numpy or device torch tensor).
    Returns (pointer, keep-alive object)."""
    if _is_torch(x):
        import torch
        want = {np.float64: torch.float64, np.int64: torch.int64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            x = x.to(want).contiguous()
        return ctypes.c_void_p(x.data_ptr()), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return ctypes.c_void_p(a.ctypes.data), a


def _stream(stream, *arrays):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    if any(_is_torch(a) and a.is_cuda for a in arrays if a is not None):
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


class Context:
    """Owns one fcas_ctx (a prepared data segment)."""

    def __init__(self, handle, setup):
        self.handle = handle
        self.setup = setup

    def close(self):
        if self.handle:
            load_library().fcas_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


FCAS_SETUP_LAZY_SCRATCH = 1


def fcas_create(det, psd, data, n_fft, fs, f_low, f_high, precision="fp32", max_batch=0, stream=None, flags=0,
                shifts=None):
    """Prepare a data segment. det: (D, 9) ECEF r, x arm, y arm; psd: (D, n_fft/2+1), or None for the
    library's analytic aLIGO fit; data: (D, n_samples).
    shifts: optional (D,) circular time shifts in samples (fcas_create_time_shifted)."""
    lib = load_library()
    det = np.asarray(det, dtype=np.float64).reshape(-1, 9)
    n_det = det.shape[0]
    dets = (fcas_detector * n_det)()
    for i in range(n_det):
        dets[i].r[:] = det[i, 0:3]
        dets[i].xarm[:] = det[i, 3:6]
        dets[i].yarm[:] = det[i, 6:9]
    n_samples = int(data.shape[-1])
    prec = ({"fp32": FCAS_PREC_FP32, "fp64": FCAS_PREC_FP64, "ff": FCAS_PREC_FF}[precision] if isinstance(precision, str)
            else int(precision))
    setup = fcas_setup(n_det, prec, n_samples, int(n_fft), float(fs), float(f_low), float(f_high), int(max_batch),
                       int(flags))
    p_psd, k1 = (ctypes.c_void_p(None), None) if psd is None else _ptr(psd, np.float64)
    p_data, k2 = _ptr(data, np.float64)
    handle = ctypes.c_void_p()
    if shifts is None:
        _check(lib.fcas_create(ctypes.byref(handle), ctypes.byref(setup), dets, p_psd, p_data,
                               _stream(stream, psd, data)))
    else:
        sh = np.asarray(shifts, dtype=np.int64).reshape(-1)
        if sh.size != n_det:
            raise ValueError(f"shifts must have one entry per detector ({n_det})")
        arr = (ctypes.c_int64 * n_det)(*[int(v) for v in sh])
        _check(lib.fcas_create_time_shifted(ctypes.byref(handle), ctypes.byref(setup), dets, p_psd, p_data, arr,
                                            _stream(stream, psd, data)))
    return Context(handle, setup)


def fcas_fitness(ctx, theta, fitness=None, tc=None, stream=None):
    """Gamma^2 and argmax t_c of a batch of particles theta (n, 4) = (alpha, delta, tau0, tau1.5).
    Outputs default to the memory kind of theta (numpy on host, torch on its CUDA device)."""
    lib = load_library()
    n = int(theta.shape[0]) if len(theta.shape) == 2 else int(np.prod(theta.shape)) // 4
    if fitness is None or tc is None:
        if _is_torch(theta) and theta.is_cuda:
            import torch
            fitness = torch.empty(n, dtype=torch.float64, device=theta.device) if fitness is None else fitness
            tc = torch.empty(n, dtype=torch.int64, device=theta.device) if tc is None else tc
        else:
            fitness = np.empty(n, dtype=np.float64) if fitness is None else fitness
            tc = np.empty(n, dtype=np.int64) if tc is None else tc
    p_th, k1 = _ptr(theta, np.float64)
    p_f, k2 = _ptr(fitness, np.float64)
    p_t, k3 = _ptr(tc, np.int64)
    _check(lib.fcas_fitness(ctx.handle, n, p_th, p_f, p_t, _stream(stream, theta, fitness, tc)))
    if k2 is not fitness and _is_torch(fitness):
        fitness.copy_(k2)
    if k3 is not tc and _is_torch(tc):
        tc.copy_(k3)
    return (k2 if not _is_torch(fitness) else fitness), (k3 if not _is_torch(tc) else tc)


def array_desc(a):
    """(is a CUDA tensor, dtype name, contiguous, device index, shape) of an argument."""
    if _is_torch(a):
        return (bool(a.is_cuda), str(a.dtype).replace("torch.", ""), bool(a.is_contiguous()),
                a.device.index if a.is_cuda else None, tuple(a.shape))
    a = np.asarray(a)
    return (False, str(a.dtype), bool(a.flags["C_CONTIGUOUS"]), None, tuple(a.shape))


def check_noalloc_arrays(theta, fitness, tc, current_device):
    """The argument checks of fcas_fitness_noalloc that the library cannot make itself (it does not
    see the arrays' sizes): theta (n, 4) float64, fitness (>= n elements) float64 and tc (>= n) int64,
    all contiguous and on the CUDA device `current_device` (the context's device, current for the
    call). Arguments are array_desc tuples. Returns n."""
    for (cuda, dtype, contiguous, dev, _), name, want in ((theta, "theta", "float64"), (fitness, "fitness", "float64"),
                                                          (tc, "tc", "int64")):
        if not (cuda and dtype == want and contiguous):
            raise TypeError(f"fcas_fitness_noalloc: {name} must be a contiguous CUDA tensor of {want}")
        if dev != current_device:
            raise ValueError(f"fcas_fitness_noalloc: {name} is on cuda:{dev} but cuda:{current_device} is current")
    shape = theta[4]
    if len(shape) != 2 or shape[1] != 4:
        raise ValueError(f"fcas_fitness_noalloc: theta must have shape (n, 4), not {shape}")
    n = int(shape[0])
    size = lambda d: int(np.prod(d[4], dtype=np.int64))
    if size(fitness) < n or size(tc) < n:
        raise ValueError(f"fcas_fitness_noalloc: fitness and tc need {n} elements, have {size(fitness)} and {size(tc)}")
    return n


def fcas_fitness_noalloc(ctx, theta, fitness, tc, stream=None):
    """Allocation-free evaluation: theta (n, 4), fitness (n,) and tc (n,) must be contiguous torch
    CUDA tensors (float64, float64, int64) on the current device, which must be the context's.
    Scratch comes from the library's fixed static device array."""
    import torch
    n = check_noalloc_arrays(array_desc(theta), array_desc(fitness), array_desc(tc), torch.cuda.current_device())
    _check(load_library().fcas_fitness_noalloc(ctx.handle, n, ctypes.c_void_p(theta.data_ptr()),
                                               ctypes.c_void_p(fitness.data_ptr()), ctypes.c_void_p(tc.data_ptr()),
                                               _stream(stream, theta, fitness, tc)))
    return fitness, tc


def fcas_destroy(ctx):
    ctx.close()


def fcas_get_info(ctx):
    info = fcas_info()
    _check(load_library().fcas_get_info(ctx.handle, ctypes.byref(info)))
    return {f: (list(getattr(info, f)) if f == "sigma2" else getattr(info, f)) for f, _ in fcas_info._fields_}


def fcas_profile_enable(ctx, on=True):
    _check(load_library().fcas_profile_enable(ctx.handle, 1 if on else 0))


def fcas_profile_read(ctx, kind):
    total = ctypes.c_double()
    launches = ctypes.c_int64()
    k = KERNEL_KINDS[kind] if isinstance(kind, str) else int(kind)
    _check(load_library().fcas_profile_read(ctx.handle, k, ctypes.byref(total), ctypes.byref(launches)))
    return total.value, launches.value


def pso_config(n_runs=8, n_particles=40, n_iter=2000, n_neighbours=1, seed=0, box=None, w_start=0.9, w_end=0.4,
               c1=2.0, c2=2.0, vmax=0.5):
    """fcas_pso_config; box = (alpha lo, hi, delta lo, hi, tau0 lo, hi, tau1.5 lo, hi)."""
    cfg = fcas_pso_config()
    cfg.n_runs, cfg.n_particles, cfg.n_iter, cfg.n_neighbours = n_runs, n_particles, n_iter, n_neighbours
    cfg.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    cfg.box[:] = [float(b) for b in box]
    cfg.w_start, cfg.w_end, cfg.c1, cfg.c2, cfg.vmax = w_start, w_end, c1, c2, vmax
    return cfg


def _check_swarm(cfg, x=(), flat=()):
    """The device kernels address n_runs x n_particles rows: every (rows, 4) float64 array in x and
    every (rows,) array in flat must be a contiguous CUDA tensor of exactly that size."""
    rows = int(cfg.n_runs) * int(cfg.n_particles)
    for t, shape in [(t, (rows, 4)) for t in x] + [(t, (rows,)) for t in flat]:
        if not (_is_torch(t) and t.is_cuda and t.is_contiguous() and tuple(t.shape) == shape and t.element_size() == 8):
            raise FcasError(-1, f"swarm arrays must be contiguous 8-byte CUDA tensors of shape {shape} "
                                f"(n_runs x n_particles = {rows} rows)")


def pso_theta(cfg, x, theta=None, stream=None):
    """Parameters of normalised positions x (torch CUDA (rows, 4)) by the library's kernel; NaN outside
    the box (not evaluated)."""
    import torch
    if theta is None:
        theta = torch.empty_like(x)
    _check_swarm(cfg, x=(x, theta))
    _check(load_library().fcas_pso_theta(ctypes.byref(cfg), ctypes.c_void_p(x.data_ptr()),
                                         ctypes.c_void_p(theta.data_ptr()), _stream(stream, x)))
    return theta


def _state(x, v, pbest_x, pbest_f, pbest_tc):
    return fcas_pso_state(*(ctypes.c_void_p(t.data_ptr()) for t in (x, v, pbest_x, pbest_f, pbest_tc)))


def fcas_pso_init(cfg, x, v, pbest_x, pbest_f, pbest_tc, stream=None):
    """Initialise device state tensors (torch CUDA, float64 / int64, rows = n_runs * n_particles)."""
    _check_swarm(cfg, x=(x, v, pbest_x), flat=(pbest_f, pbest_tc))
    st = _state(x, v, pbest_x, pbest_f, pbest_tc)
    _check(load_library().fcas_pso_init(ctypes.byref(cfg), ctypes.byref(st), _stream(stream, x)))


def fcas_pso_update(cfg, it, fitness, tc, x, v, pbest_x, pbest_f, pbest_tc, stream=None):
    _check_swarm(cfg, x=(x, v, pbest_x), flat=(pbest_f, pbest_tc, fitness, tc))
    st = _state(x, v, pbest_x, pbest_f, pbest_tc)
    _check(load_library().fcas_pso_update(ctypes.byref(cfg), int(it), ctypes.c_void_p(fitness.data_ptr()),
                                          ctypes.c_void_p(tc.data_ptr()), ctypes.byref(st), _stream(stream, x)))


def pso_save(path, cfg, it, x, v, pbest_x, pbest_f, pbest_tc):
    """Checkpoint: the swarm state after iteration `it` (tensors or arrays) and its configuration, as
    an .npz file written atomically (a temporary file, then a rename)."""
    arrays = {k: (t.detach().cpu().numpy() if _is_torch(t) else np.asarray(t))
              for k, t in zip(("x", "v", "pbest_x", "pbest_f", "pbest_tc"), (x, v, pbest_x, pbest_f, pbest_tc))}
    tmp = path + ".tmp.npz"
    np.savez(tmp, it=np.int64(it), cfg=np.frombuffer(bytes(cfg), dtype=np.uint8), **arrays)
    os.replace(tmp, path)


def pso_load(path, device=None):
    """Read a checkpoint: (cfg, it, [x, v, pbest_x, pbest_f, pbest_tc]); the state as torch tensors on
    `device`, or numpy arrays when device is None."""
    with np.load(path) as z:
        cfg = fcas_pso_config.from_buffer_copy(z["cfg"].tobytes())
        it = int(z["it"])
        state = [z[k].copy() for k in ("x", "v", "pbest_x", "pbest_f", "pbest_tc")]
    if device is not None:
        import torch
        state = [torch.from_numpy(a).to(device) for a in state]
    return cfg, it, state


def pso_run(ctx, cfg, checkpoint=None, every=0, resume=False, stop_after=None, device="cuda:0"):
    """The PSO search iteration by iteration through fcas_pso_theta / fcas_fitness / fcas_pso_update
    (the same steps as fcas_search, without its graph replay), checkpointing the swarm to
    `checkpoint` every `every` iterations and, with resume=True, continuing from the checkpoint when
    one exists (its configuration must equal cfg). The counter-based random numbers make a resumed
    run identical to an uninterrupted one. stop_after ends the run after that many iterations of this
    call (an interruption). Returns (results per run as fcas_search reports them, iterations done)."""
    import torch
    rows = cfg.n_runs * cfg.n_particles
    start = 0
    if resume and checkpoint and os.path.exists(checkpoint):
        saved_cfg, it, state = pso_load(checkpoint, device)
        if bytes(saved_cfg) != bytes(cfg):
            raise FcasError(-1, "pso_run: the checkpoint was written for another configuration")
        start = it + 1
    else:
        x = torch.empty((rows, 4), dtype=torch.float64, device=device)
        state = [x, torch.empty_like(x), torch.empty_like(x), torch.empty(rows, dtype=torch.float64, device=device),
                 torch.empty(rows, dtype=torch.int64, device=device)]
        fcas_pso_init(cfg, *state)
    stop = cfg.n_iter if stop_after is None else min(cfg.n_iter, start + int(stop_after))
    it = start - 1
    for it in range(start, stop):
        theta = pso_theta(cfg, state[0])
        fit, tc = fcas_fitness(ctx, theta)
        fcas_pso_update(cfg, it, fit, tc, *state)
        if checkpoint and every and ((it + 1) % every == 0 or it + 1 == cfg.n_iter):
            pso_save(checkpoint, cfg, it, *state)
    pbest_f = state[3].view(cfg.n_runs, cfg.n_particles)
    best = torch.argmax(torch.nan_to_num(pbest_f, nan=-np.inf), dim=1)   # first maximum of each run
    idx = torch.arange(cfg.n_runs, device=pbest_f.device) * cfg.n_particles + best
    theta = pso_theta(cfg, state[2])[idx].cpu().numpy()   # the kernel maps all n_runs x n_particles rows
    f, t = state[3][idx].cpu().numpy(), state[4][idx].cpu().numpy()
    res = [dict(fitness=float(f[r]), theta=list(theta[r]), tc=int(t[r])) for r in range(cfg.n_runs)]
    return res, it + 1


def fcas_search(ctx, cfg, stream=None):
    """Run the device PSO search; returns a list of dicts (one per run)."""
    res = (fcas_search_result * cfg.n_runs)()
    s = ctypes.c_void_p(int(stream)) if stream is not None else ctypes.c_void_p(0)
    _check(load_library().fcas_search(ctx.handle, ctypes.byref(cfg), res, s))
    return [dict(fitness=r.fitness, theta=list(r.theta), tc=r.tc, evaluations=r.evaluations) for r in res]


def fcas_gradient(ctx, theta, tc, grad=None, stream=None):
    """d Gamma^2 / d theta at fixed tc (n, 4); output follows theta's memory kind unless given."""
    n = int(theta.shape[0])
    if grad is None:
        if _is_torch(theta) and theta.is_cuda:
            import torch
            grad = torch.empty((n, 4), dtype=torch.float64, device=theta.device)
        else:
            grad = np.empty((n, 4), dtype=np.float64)
    p_th, k1 = _ptr(theta, np.float64)
    p_tc, k2 = _ptr(tc, np.int64)
    p_g, k3 = _ptr(grad, np.float64)
    _check(load_library().fcas_gradient(ctx.handle, n, p_th, p_tc, p_g, _stream(stream, theta, tc, grad)))
    if k3 is not grad and _is_torch(grad):
        grad.copy_(k3)
    return k3 if not _is_torch(grad) else grad


def _autograd_function():
    import torch

    class CoherentFitness(torch.autograd.Function):
        """Gamma^2(theta) with its adjoint: forward = fcas_fitness, backward = fcas_gradient at the
        forward pass's argmax t_c (the maximisation over t_c is held fixed)."""

        @staticmethod
        def forward(actx, theta, fctx):
            fit, tc = fcas_fitness(fctx, theta.detach().contiguous())
            actx.save_for_backward(theta, tc)
            actx.fctx = fctx
            actx.mark_non_differentiable(tc)
            return fit, tc

        @staticmethod
        def backward(actx, g_fit, g_tc):
            theta, tc = actx.saved_tensors
            grad = fcas_gradient(actx.fctx, theta.detach().contiguous(), tc)
            return grad * g_fit.unsqueeze(1), None

    return CoherentFitness


_CF = None


def coherent_fitness(ctx, theta):
    """Differentiable fitness for torch CUDA tensors: returns (fitness, tc); fitness.backward()
    propagates d Gamma^2 / d theta through the library's adjoint kernel."""
    global _CF
    if _CF is None:
        _CF = _autograd_function()
    return _CF.apply(theta, ctx)


def fcas_polish(ctx, theta, steps=10, scales=(1e-2, 1e-2, 1e-4, 1e-4), max_halvings=30, stream=None):
    """Gradient polishing by the library (C: fcas_polish) of points theta (n, 4), numpy or a torch
    CUDA tensor (updated in place when it is a contiguous float64 CUDA tensor). Returns (theta,
    fitness, tc, accepted steps), each in theta's memory kind."""
    n = int(theta.shape[0])
    if _is_torch(theta) and theta.is_cuda:
        import torch
        th = theta if (theta.dtype == torch.float64 and theta.is_contiguous()) else theta.to(torch.float64).contiguous()
        fit = torch.empty(n, dtype=torch.float64, device=theta.device)
        tc = torch.empty(n, dtype=torch.int64, device=theta.device)
        acc = torch.empty(n, dtype=torch.int32, device=theta.device)
        ptrs = [ctypes.c_void_p(t.data_ptr()) for t in (th, fit, tc, acc)]
    else:
        th = np.array(theta, dtype=np.float64).reshape(n, 4)
        fit, tc, acc = np.empty(n), np.empty(n, dtype=np.int64), np.empty(n, dtype=np.int32)
        ptrs = [ctypes.c_void_p(a.ctypes.data) for a in (th, fit, tc, acc)]
    sc = (ctypes.c_double * 4)(*[float(v) for v in scales])
    _check(load_library().fcas_polish(ctx.handle, n, ptrs[0], ptrs[1], ptrs[2], int(steps), sc, int(max_halvings),
                                      ptrs[3], _stream(stream, theta)))
    return th, fit, tc, acc


def fcas_autotune(ctx, n_particles=64, cache_path=None, stream=None):
    """Time the launch shapes on this context and keep the fastest; returns fcas_get_info(ctx)."""
    path = cache_path.encode() if cache_path else None
    s = ctypes.c_void_p(int(stream)) if stream is not None else ctypes.c_void_p(0)
    _check(load_library().fcas_autotune(ctx.handle, int(n_particles), path, s))
    return fcas_get_info(ctx)


def fcas_set_shape(ctx, split_bias=0, k1b=0, sub=8, radix_bits_a=4, stream=None):
    s = ctypes.c_void_p(int(stream)) if stream is not None else ctypes.c_void_p(0)
    _check(load_library().fcas_set_shape(ctx.handle, int(split_bias), int(k1b), int(sub), int(radix_bits_a), s))
    return fcas_get_info(ctx)


class Group:
    """Owns one fcas_group (segments searched together with shared scratch)."""

    def __init__(self, contexts, max_batch=0):
        self.contexts = list(contexts)           # keep the contexts alive as long as the group
        arr = (ctypes.c_void_p * len(self.contexts))(*[c.handle for c in self.contexts])
        self.handle = ctypes.c_void_p()
        _check(load_library().fcas_group_create(ctypes.byref(self.handle), len(self.contexts), arr, int(max_batch)))

    def search(self, cfg, stream=None, boxes=None):
        """Returns a list (per segment) of lists (per run) of result dicts. boxes: optional (n_ctx, 8)
        PSO box per segment (fcas_group_search_boxes)."""
        n = len(self.contexts)
        res = (fcas_search_result * (n * cfg.n_runs))()
        s = ctypes.c_void_p(int(stream)) if stream is not None else ctypes.c_void_p(0)
        if boxes is None:
            _check(load_library().fcas_group_search(self.handle, ctypes.byref(cfg), res, s))
        else:
            b = np.ascontiguousarray(np.asarray(boxes, dtype=np.float64).reshape(-1))
            if b.size != 8 * n:
                raise ValueError(f"boxes must be ({n}, 8)")
            _check(load_library().fcas_group_search_boxes(self.handle, ctypes.byref(cfg),
                                                          b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), res, s))
        out = [dict(fitness=r.fitness, theta=list(r.theta), tc=r.tc, evaluations=r.evaluations) for r in res]
        return [out[i * cfg.n_runs:(i + 1) * cfg.n_runs] for i in range(n)]

    def close(self):
        if self.handle:
            load_library().fcas_group_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def fcas_group_create(contexts, max_batch=0):
    return Group(contexts, max_batch)


def segment_seed(seed, s):
    """Key of segment s's swarm in a group search (seed + s * 0x9E3779B97F4A7C15 mod 2^64)."""
    return (int(seed) + s * 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF


def fcas_tau_tiles(tau0_lo, tau0_hi, tau15_lo, tau15_hi, n0, n15, overlap=0.0):
    """(n0 * n15, 8) PSO boxes over the whole sky tiling the chirp-time rectangle with the given
    overlap fraction (C: fcas_tau_tiles; host only)."""
    out = np.zeros((int(n0) * int(n15), 8))
    _check(load_library().fcas_tau_tiles(float(tau0_lo), float(tau0_hi), float(tau15_lo), float(tau15_hi), int(n0),
                                         int(n15), float(overlap), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def time_slide_background(det, psd, data, n_fft, fs, f_low, f_high, shifts, cfg, precision="fp32", max_batch=0,
                          stream=None):
    """Background of the search statistic from time-shifted copies of one data realisation (Sec. V):
    one context per row of shifts (S, D) (fcas_create_time_shifted, lazy scratch), all searched
    together by one group with cfg. Returns (best fitness per slide (S,), per-slide run results)."""
    ctxs = [fcas_create(det, psd, data, n_fft, fs, f_low, f_high, precision=precision, stream=stream,
                        flags=FCAS_SETUP_LAZY_SCRATCH, shifts=row) for row in np.asarray(shifts)]
    try:
        with Group(ctxs, max_batch=max_batch) as g:
            res = g.search(cfg, stream=stream)
    finally:
        for c in ctxs:
            c.close()
    best = np.array([max(r["fitness"] for r in seg) for seg in res])
    return best, res


def fcas_condition_number(ctx, theta, kappa=None, stream=None):
    """Condition number of the antenna-pattern matrix at each particle's (alpha, delta) (C:
    fcas_condition_number). Output defaults to the memory kind of theta."""
    n = int(theta.shape[0]) if len(theta.shape) == 2 else int(np.prod(theta.shape)) // 4
    if kappa is None:
        if _is_torch(theta) and theta.is_cuda:
            import torch
            kappa = torch.empty(n, dtype=torch.float64, device=theta.device)
        else:
            kappa = np.empty(n, dtype=np.float64)
    p_th, k1 = _ptr(theta, np.float64)
    p_k, k2 = _ptr(kappa, np.float64)
    _check(load_library().fcas_condition_number(ctx.handle, n, p_th, p_k, _stream(stream, theta, kappa)))
    return kappa
